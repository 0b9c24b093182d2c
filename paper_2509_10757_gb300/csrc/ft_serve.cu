// ft_serve.cu -- the served request loop: continuous batching of tracking
// requests from many camera streams on one GPU.
//
// Streams are admitted against an HBM budget: the server preallocates one
// device pool of that size and gives each admitted stream a block holding its
// resident state (both pyramids, the local map, the per-frame keypoint block
// and the output block).  A request carries one frame's keypoints, taken
// flags and pose in host memory, and optionally the frame's two level-0
// images; submit packs them into the stream's pinned staging buffers.  A
// request with images replaces the resident level 0 at launch, and the batch
// rebuilds that stream's levels 1.. on the device before it matches.  A scheduler thread fills free slots (a slot = an ft_ctx
// with its own arena and CUDA stream) with batches of pending requests, at
// most one per stream, in arrival order: one host-to-device copy per
// request, one ft_track_batch launch per batch, one device-to-host copy of
// each request's results, and a host function on the stream that timestamps
// the batch's completion.  Requests that arrive while a batch runs are taken
// by the next free slot, so batches overlap on the device.
//
// A dry-run server (no GPU) replaces the device work by a fake completion
// after a fixed delay; it exercises the same admission and scheduling code.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "ft_internal.h"

using namespace ft;

namespace {

double now_us()
{
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

ft_status fail(ft_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

size_t al16(size_t v) { return (v + 15) / 16 * 16; }
size_t al256(size_t v) { return (v + 255) / 256 * 256; }

// First-fit allocator over [0, capacity) of the server's device pool.
class Pool {
  public:
    explicit Pool(size_t cap) : cap_(cap) { free_.push_back({0, cap}); }
    bool alloc(size_t size, size_t *off)
    {
        size = al256(std::max<size_t>(size, 1));
        for (size_t i = 0; i < free_.size(); ++i) {
            if (free_[i].size >= size) {
                *off = free_[i].off;
                free_[i].off += size;
                free_[i].size -= size;
                if (free_[i].size == 0) free_.erase(free_.begin() + (long)i);
                used_ += size;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t size)
    {
        size = al256(std::max<size_t>(size, 1));
        used_ -= size;
        auto it = std::lower_bound(free_.begin(), free_.end(), off,
                                   [](const Blk &b, size_t o) { return b.off < o; });
        it = free_.insert(it, {off, size});
        size_t i = (size_t)(it - free_.begin());
        if (i + 1 < free_.size() && free_[i].off + free_[i].size == free_[i + 1].off) {
            free_[i].size += free_[i + 1].size;
            free_.erase(free_.begin() + (long)i + 1);
        }
        if (i > 0 && free_[i - 1].off + free_[i - 1].size == free_[i].off) {
            free_[i - 1].size += free_[i].size;
            free_.erase(free_.begin() + (long)i);
        }
    }
    size_t used() const { return used_; }
    size_t capacity() const { return cap_; }

  private:
    struct Blk {
        size_t off, size;
    };
    size_t cap_, used_ = 0;
    std::vector<Blk> free_;
};

// Compact layout of a request's keypoint block (host staging and device) and
// of its result block; offsets depend on this request's counts.
struct DynLayout {
    size_t lx, ly, loct, ldesc, rx, ry, roct, rdesc, tl, tr, bytes;
};
DynLayout dyn_layout(int nl, int nr)
{
    DynLayout L{};
    size_t o = 0;
    auto put = [&](size_t &f, size_t b) {
        f = o;
        o = al16(o + b);
    };
    put(L.lx, 4 * (size_t)nl);
    put(L.ly, 4 * (size_t)nl);
    put(L.loct, (size_t)nl);
    put(L.ldesc, 32 * (size_t)nl);
    put(L.rx, 4 * (size_t)nr);
    put(L.ry, 4 * (size_t)nr);
    put(L.roct, (size_t)nr);
    put(L.rdesc, 32 * (size_t)nr);
    put(L.tl, (size_t)nl);
    put(L.tr, (size_t)nr);
    L.bytes = o;
    return L;
}

struct OutLayout {
    size_t st[6];                  // best_r, dist, sad_shift, sad_best, u_right, depth (pinhole)
    size_t fo[5];                  // r_idx, d1, d2, depth, xyz (fisheye)
    size_t cam[2][6];              // level, proj, mp_kp, mp_d1, mp_d2, kp_mp per camera
    size_t bytes;
};
OutLayout out_layout(int camera, int nl, int nr, int m)
{
    OutLayout L{};
    size_t o = 0;
    auto put = [&](size_t &f, size_t b) {
        f = o;
        o = al16(o + b);
    };
    if (camera == FT_CAMERA_PINHOLE) {
        for (int k = 0; k < 6; ++k) put(L.st[k], 4 * (size_t)nl);
    } else {
        for (int k = 0; k < 4; ++k) put(L.fo[k], 4 * (size_t)nl);
        put(L.fo[4], 16 * (size_t)nl);
    }
    const int ncam = camera == FT_CAMERA_FISHEYE ? 2 : 1;
    for (int c = 0; c < ncam; ++c) {
        put(L.cam[c][0], (size_t)m);
        put(L.cam[c][1], 16 * (size_t)m);
        for (int k = 2; k < 5; ++k) put(L.cam[c][k], 4 * (size_t)m);
        put(L.cam[c][5], 4 * (size_t)(c ? nr : nl));
    }
    L.bytes = o;
    return L;
}

constexpr int kMaxQueue = 8;       // waiting requests a stream may be configured for, at most

struct StreamState {
    bool open = false;
    ft_stream_desc desc{};
    size_t off = 0, bytes = 0;     // block in the pool
    char *dev = nullptr;           // base of the block
    size_t o_pyrL[FT_MAX_LEVELS] = {}, o_pyrR[FT_MAX_LEVELS] = {};
    size_t o_pos = 0, o_nrm = 0, o_mdesc = 0, o_skip = 0, o_dyn = 0, o_out = 0;
    int map_n = 0;
    char *h_dyn[kMaxQueue] = {};   // pinned staging of the waiting requests (queue_depth of them)
    int dyn_used[kMaxQueue] = {};
    char *h_out[2] = {nullptr, nullptr};   // pinned copies of two results (one request runs at a time)
    char *h_img[kMaxQueue] = {};   // pinned level-0 images of the waiting requests (left, then right;
                                   // allocated at the first request that carries images)
    int next_out = 0;
    bool in_flight = false;
    int queued = 0;
};

struct Request {
    uint64_t tag = 0;
    int sid = -1, buf = 0, nl = 0, nr = 0;
    bool images = false;           // level-0 images staged in h_img[buf]
    ft_pose pose{};
    float O_right[3] = {0, 0, 0};
    double t_submit = 0;
    int out_buf = 0;
};

struct Slot;
struct DoneArg {
    ft_server *server;
    Slot *slot;
};

struct Slot {
    ft_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<Request> reqs;
    bool busy = false;
    std::atomic<int> done{0};
    double t_start = 0, t_done = 0;
    DoneArg arg{};
};

void CUDART_CB host_done(void *p);

}  // namespace

struct ft_server {
    ft_server_desc desc{};
    ft_params params{};
    bool dry = false;
    int depth = 2;                     // requests a stream may have waiting
    char *pool_mem = nullptr;
    Pool *pool = nullptr;
    std::deque<StreamState> streams;   // a deque: references stay valid while streams open
    std::vector<Slot *> slots;
    std::mutex mu;
    std::condition_variable cv;        // scheduler wake-up
    std::condition_variable done_cv;   // completions available
    std::deque<Request> pending;
    std::deque<ft_completion> completed;
    std::thread thread;
    bool stop = false;
    ft_server_stats stats{};
    ft_status last_launch_status = FT_OK;
};

namespace {

// The pinned staging of a stream (null entries skipped).
void free_staging(StreamState &S)
{
    for (int b = 0; b < kMaxQueue; ++b) {
        if (S.h_dyn[b]) cudaFreeHost(S.h_dyn[b]);
        if (S.h_img[b]) cudaFreeHost(S.h_img[b]);
        S.h_dyn[b] = S.h_img[b] = nullptr;
    }
    for (int b = 0; b < 2; ++b) {
        if (S.h_out[b]) cudaFreeHost(S.h_out[b]);
        S.h_out[b] = nullptr;
    }
}

void CUDART_CB host_done(void *p)
{
    DoneArg *a = static_cast<DoneArg *>(p);
    a->slot->t_done = now_us();
    {
        std::lock_guard<std::mutex> lk(a->server->mu);
        a->slot->done.store(1);
    }
    a->server->cv.notify_one();
}

// resident pyramid rows are padded to 16 bytes (the kernel reads 4-byte words)
size_t level_pitch(const ft_stream_desc &d, int l) { return al16((size_t)d.level_width[l]); }

size_t stream_block_bytes(const ft_stream_desc &d, ft_params const &p, StreamState *S)
{
    size_t o = 0;
    auto put = [&](size_t &f, size_t b) {
        f = o;
        o = al256(o + b);
    };
    size_t dummy;
    if (d.camera == FT_CAMERA_PINHOLE) {
        for (int l = 0; l < p.nlevels; ++l) put(S ? S->o_pyrL[l] : dummy, level_pitch(d, l) * d.level_height[l]);
        for (int l = 0; l < p.nlevels; ++l) put(S ? S->o_pyrR[l] : dummy, level_pitch(d, l) * d.level_height[l]);
    }
    put(S ? S->o_pos : dummy, 16 * (size_t)d.max_map);
    put(S ? S->o_nrm : dummy, 16 * (size_t)d.max_map);
    put(S ? S->o_mdesc : dummy, 32 * (size_t)d.max_map);
    put(S ? S->o_skip : dummy, (size_t)d.max_map);
    put(S ? S->o_dyn : dummy, dyn_layout(d.max_left, d.max_right).bytes);
    put(S ? S->o_out : dummy, out_layout(d.camera, d.max_left, d.max_right, d.max_map).bytes);
    return o;
}

ft_results results_of(const StreamState &S, const Request &r, const char *base)
{
    ft_results R{};
    R.n_left = r.nl;
    R.n_right = r.nr;
    R.n_map = S.map_n;
    const OutLayout O = out_layout(S.desc.camera, r.nl, r.nr, S.map_n);
    auto at = [&](size_t off) { return const_cast<char *>(base) + off; };
    if (S.desc.camera == FT_CAMERA_PINHOLE) {
        R.stereo.best_r = reinterpret_cast<int32_t *>(at(O.st[0]));
        R.stereo.dist = reinterpret_cast<int32_t *>(at(O.st[1]));
        R.stereo.sad_shift = reinterpret_cast<int32_t *>(at(O.st[2]));
        R.stereo.sad_best = reinterpret_cast<int32_t *>(at(O.st[3]));
        R.stereo.u_right = reinterpret_cast<float *>(at(O.st[4]));
        R.stereo.depth = reinterpret_cast<float *>(at(O.st[5]));
    } else {
        R.fisheye.r_idx = reinterpret_cast<int32_t *>(at(O.fo[0]));
        R.fisheye.d1 = reinterpret_cast<int32_t *>(at(O.fo[1]));
        R.fisheye.d2 = reinterpret_cast<int32_t *>(at(O.fo[2]));
        R.fisheye.depth = reinterpret_cast<float *>(at(O.fo[3]));
        R.fisheye.xyz = reinterpret_cast<float *>(at(O.fo[4]));
    }
    const int ncam = S.desc.camera == FT_CAMERA_FISHEYE ? 2 : 1;
    for (int c = 0; c < ncam; ++c) {
        ft_search_cam_out &o = c ? R.search.right : R.search.left;
        o.level = reinterpret_cast<int8_t *>(at(O.cam[c][0]));
        o.proj = reinterpret_cast<float *>(at(O.cam[c][1]));
        o.mp_kp = reinterpret_cast<int32_t *>(at(O.cam[c][2]));
        o.mp_d1 = reinterpret_cast<int32_t *>(at(O.cam[c][3]));
        o.mp_d2 = reinterpret_cast<int32_t *>(at(O.cam[c][4]));
        o.kp_mp = reinterpret_cast<int32_t *>(at(O.cam[c][5]));
    }
    return R;
}

// The device-side frame job of a request (resident state + its keypoint block).
ft_frame_job job_of(const StreamState &S, const Request &r)
{
    ft_frame_job j{};
    const ft_stream_desc &d = S.desc;
    j.camera = d.camera;
    j.pinhole = d.pinhole;
    j.fisheye = d.fisheye;
    const DynLayout D = dyn_layout(r.nl, r.nr);
    char *dyn = S.dev + S.o_dyn;
    j.left = ft_keypoints{r.nl, reinterpret_cast<float *>(dyn + D.lx), reinterpret_cast<float *>(dyn + D.ly),
                          reinterpret_cast<int8_t *>(dyn + D.loct), reinterpret_cast<uint8_t *>(dyn + D.ldesc)};
    j.right = ft_keypoints{r.nr, reinterpret_cast<float *>(dyn + D.rx), reinterpret_cast<float *>(dyn + D.ry),
                           reinterpret_cast<int8_t *>(dyn + D.roct), reinterpret_cast<uint8_t *>(dyn + D.rdesc)};
    j.taken_left = reinterpret_cast<uint8_t *>(dyn + D.tl);
    j.taken_right = reinterpret_cast<uint8_t *>(dyn + D.tr);
    if (d.camera == FT_CAMERA_PINHOLE) {
        j.pyr_left.nlevels = j.pyr_right.nlevels = d.nlevels;
        for (int l = 0; l < d.nlevels; ++l) {
            j.pyr_left.data[l] = reinterpret_cast<uint8_t *>(S.dev + S.o_pyrL[l]);
            j.pyr_right.data[l] = reinterpret_cast<uint8_t *>(S.dev + S.o_pyrR[l]);
            j.pyr_left.width[l] = j.pyr_right.width[l] = d.level_width[l];
            j.pyr_left.height[l] = j.pyr_right.height[l] = d.level_height[l];
            j.pyr_left.pitch[l] = j.pyr_right.pitch[l] = (int)level_pitch(d, l);
        }
    }
    j.build_pyramids = r.images ? 1 : 0;
    j.pose = r.pose;
    for (int i = 0; i < 3; ++i) j.O_right[i] = r.O_right[i];
    j.map = ft_map_view{S.map_n, reinterpret_cast<float *>(S.dev + S.o_pos), reinterpret_cast<float *>(S.dev + S.o_nrm),
                        reinterpret_cast<uint8_t *>(S.dev + S.o_mdesc), reinterpret_cast<uint8_t *>(S.dev + S.o_skip)};
    const ft_results R = results_of(S, r, S.dev + S.o_out);
    j.stereo = R.stereo;
    j.fisheye_out = R.fisheye;
    j.search = R.search;
    return j;
}

// Launch one batch on a free slot (scheduler thread, lock not held).
ft_status launch(ft_server *s, Slot &sl)
{
    sl.t_start = now_us();
    if (s->dry) {
        // fake completion: the batch "finishes" after the configured delay
        sl.t_done = sl.t_start + s->desc.dry_run_latency_us;
        sl.done.store(1);
        return FT_OK;
    }
    std::vector<ft_frame_job> jobs;
    jobs.reserve(sl.reqs.size());
    for (Request &r : sl.reqs) {
        StreamState &S = s->streams[r.sid];
        const DynLayout D = dyn_layout(r.nl, r.nr);
        if (cudaMemcpyAsync(S.dev + S.o_dyn, S.h_dyn[r.buf], D.bytes, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
            return fail(FT_ECUDA, "server: upload failed");
        if (r.images) {
            // the stream's previous request has completed (one in flight per
            // stream), so its level 0 may be overwritten
            const size_t b0 = level_pitch(S.desc, 0) * (size_t)S.desc.level_height[0];
            if (cudaMemcpyAsync(S.dev + S.o_pyrL[0], S.h_img[r.buf], b0, cudaMemcpyHostToDevice, sl.stream) !=
                    cudaSuccess ||
                cudaMemcpyAsync(S.dev + S.o_pyrR[0], S.h_img[r.buf] + b0, b0, cudaMemcpyHostToDevice, sl.stream) !=
                    cudaSuccess)
                return fail(FT_ECUDA, "server: image upload failed");
        }
        jobs.push_back(job_of(S, r));
    }
    ft_batch b{};
    b.n = (int)jobs.size();
    b.frames = jobs.data();
    ft_status st = ft_track_batch(sl.ctx, sl.stream, &s->params, &b);
    if (st != FT_OK) return st;
    for (Request &r : sl.reqs) {
        StreamState &S = s->streams[r.sid];
        const OutLayout O = out_layout(S.desc.camera, r.nl, r.nr, S.map_n);
        if (cudaMemcpyAsync(S.h_out[r.out_buf], S.dev + S.o_out, O.bytes, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
            return fail(FT_ECUDA, "server: download failed");
    }
    if (cudaLaunchHostFunc(sl.stream, host_done, &sl.arg) != cudaSuccess)
        return fail(FT_ECUDA, "server: cudaLaunchHostFunc failed");
    return FT_OK;
}

void scheduler(ft_server *s)
{
    if (!s->dry) cudaSetDevice(s->desc.device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        bool progress = false;
        // 1. completed batches -> completions, streams free again
        for (Slot *sl : s->slots) {
            if (!sl->busy) continue;
            if (s->dry && now_us() < sl->t_done) continue;
            if (!sl->done.load()) continue;
            for (Request &r : sl->reqs) {
                StreamState &S = s->streams[r.sid];
                ft_completion c{};
                c.tag = r.tag;
                c.stream_id = r.sid;
                c.status = FT_OK;
                c.t_submit_us = r.t_submit;
                c.t_start_us = sl->t_start;
                c.t_done_us = sl->t_done;
                if (!s->dry) c.results = results_of(S, r, S.h_out[r.out_buf]);
                else c.results.n_left = r.nl, c.results.n_right = r.nr, c.results.n_map = S.map_n;
                S.in_flight = false;
                S.dyn_used[r.buf] = 0;
                s->completed.push_back(c);
                s->stats.completed += 1;
            }
            sl->reqs.clear();
            sl->busy = false;
            sl->done.store(0);
            progress = true;
        }
        if (progress) s->done_cv.notify_all();
        // 2. free slots take pending requests: arrival order, one per stream,
        //    none of a stream whose previous request is still on the GPU
        for (Slot *sl : s->slots) {
            if (sl->busy || s->pending.empty()) continue;
            std::vector<int> taken_streams;
            for (auto it = s->pending.begin(); it != s->pending.end() && (int)sl->reqs.size() < s->desc.max_batch;) {
                StreamState &S = s->streams[it->sid];
                if (S.in_flight || std::find(taken_streams.begin(), taken_streams.end(), it->sid) != taken_streams.end()) {
                    // keep this stream's order: none of its later requests may pass
                    taken_streams.push_back(it->sid);
                    ++it;
                    continue;
                }
                Request r = *it;
                it = s->pending.erase(it);
                S.queued -= 1;
                S.in_flight = true;
                r.out_buf = S.next_out;
                S.next_out ^= 1;
                sl->reqs.push_back(r);
                taken_streams.push_back(r.sid);
            }
            if (sl->reqs.empty()) continue;
            sl->busy = true;
            sl->done.store(0);
            s->stats.batches += 1;
            s->stats.frames_launched += sl->reqs.size();
            lk.unlock();
            const ft_status st = launch(s, *sl);
            lk.lock();
            if (st != FT_OK) s->last_launch_status = st;
            progress = true;
        }
        if (!progress) s->cv.wait_for(lk, std::chrono::microseconds(s->dry ? 20 : 200));
    }
}

}  // namespace

extern "C" {

void ft_server_desc_default(ft_server_desc *d)
{
    if (!d) return;
    std::memset(d, 0, sizeof(*d));
    d->device = 0;
    d->hbm_budget = (size_t)4 << 30;
    d->n_slots = 2;
    d->max_batch = 64;
    d->slot_arena_bytes = (size_t)256 << 20;
    d->dry_run = 0;
    d->dry_run_latency_us = 100.0;
}

ft_status ft_server_create(ft_server **out, const ft_server_desc *desc, const ft_params *params)
{
    if (!out || !desc) return fail(FT_EINVAL, "ft_server_create: NULL argument");
    *out = nullptr;
    const ft_server_desc &d = *desc;
    if (d.n_slots < 1 || d.n_slots > 64 || d.max_batch < 1 || d.max_batch > 4096 || d.hbm_budget == 0)
        return fail(FT_EINVAL, "ft_server_create: bad slots / batch / budget");
    if (d.queue_depth < 0 || d.queue_depth > kMaxQueue)
        return fail(FT_EINVAL, "ft_server_create: queue depth %d outside 0-%d", d.queue_depth, kMaxQueue);
    ft_server *s = new ft_server();
    s->desc = d;
    s->depth = d.queue_depth > 0 ? d.queue_depth : 2;
    s->dry = d.dry_run != 0;
    if (params) s->params = *params;
    else ft_params_default(&s->params);
    s->pool = new Pool(d.hbm_budget);
    if (!s->dry) {
        cudaError_t e = cudaSetDevice(d.device);
        if (e == cudaSuccess) e = cudaMalloc(&s->pool_mem, d.hbm_budget);
        if (e != cudaSuccess) {
            ft_server_destroy(s);
            return fail(FT_ENOMEM, "ft_server_create: device pool of %zu bytes: %s", d.hbm_budget,
                        cudaGetErrorString(e));
        }
    }
    for (int i = 0; i < d.n_slots; ++i) {
        Slot *sl = new Slot();
        sl->arg = DoneArg{s, sl};
        s->slots.push_back(sl);
        if (!s->dry) {
            ft_ctx_desc cd{};
            cd.device = d.device;
            cd.arena_bytes = d.slot_arena_bytes;
            cd.max_frames = d.max_batch;
            cd.use_graphs = 1;
            ft_status st = ft_create(&sl->ctx, &cd);
            if (st == FT_OK && cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess)
                st = FT_ECUDA;
            if (st != FT_OK) {
                ft_server_destroy(s);
                return fail(st, "ft_server_create: slot %d could not be created", i);
            }
        }
    }
    s->thread = std::thread(scheduler, s);
    *out = s;
    return FT_OK;
}

void ft_server_destroy(ft_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->thread.joinable()) s->thread.join();
    for (Slot *sl : s->slots) {
        if (sl->stream) {
            cudaStreamSynchronize(sl->stream);
            cudaStreamDestroy(sl->stream);
        }
        if (sl->ctx) ft_destroy(sl->ctx);
        delete sl;
    }
    for (StreamState &S : s->streams) free_staging(S);
    if (s->pool_mem) cudaFree(s->pool_mem);
    delete s->pool;
    delete s;
}

ft_status ft_server_open_stream(ft_server *s, const ft_stream_desc *d, int *stream_id)
{
    if (!s || !d || !stream_id) return fail(FT_EINVAL, "ft_server_open_stream: NULL argument");
    if (d->camera != FT_CAMERA_PINHOLE && d->camera != FT_CAMERA_FISHEYE)
        return fail(FT_EINVAL, "unknown camera model %d", d->camera);
    if (d->max_left < 0 || d->max_right < 0 || d->max_map < 0 || d->max_left >= FT_MAX_KEYPOINTS ||
        d->max_right >= FT_MAX_KEYPOINTS)
        return fail(FT_EINVAL, "bad stream capacities");
    if (d->camera == FT_CAMERA_PINHOLE) {
        if (d->nlevels != s->params.nlevels) return fail(FT_EINVAL, "stream has %d levels, server %d", d->nlevels, s->params.nlevels);
        for (int l = 0; l < d->nlevels; ++l)
            if (d->level_width[l] <= 0 || d->level_height[l] <= 0) return fail(FT_EINVAL, "bad level %d size", l);
    }
    StreamState S;
    S.desc = *d;
    const size_t bytes = stream_block_bytes(*d, s->params, &S);
    std::lock_guard<std::mutex> lk(s->mu);
    size_t off = 0;
    if (!s->pool->alloc(bytes, &off))
        return fail(FT_EBUSY, "HBM budget: stream needs %zu bytes, %zu of %zu in use", bytes, s->pool->used(),
                    s->pool->capacity());
    S.off = off;
    S.bytes = bytes;
    S.dev = s->dry ? nullptr : s->pool_mem + off;
    if (!s->dry) {
        const size_t dynb = dyn_layout(d->max_left, d->max_right).bytes;
        const size_t outb = out_layout(d->camera, d->max_left, d->max_right, d->max_map).bytes;
        bool ok = true;
        for (int b = 0; b < s->depth && ok; ++b)
            ok = cudaMallocHost(&S.h_dyn[b], std::max<size_t>(dynb, 16)) == cudaSuccess;
        for (int b = 0; b < 2 && ok; ++b)
            ok = cudaMallocHost(&S.h_out[b], std::max<size_t>(outb, 16)) == cudaSuccess;
        if (!ok) {
            free_staging(S);
            s->pool->release(off, bytes);
            return fail(FT_ENOMEM, "pinned staging for the stream could not be allocated");
        }
    }
    S.open = true;
    int id = -1;
    for (size_t i = 0; i < s->streams.size(); ++i)
        if (!s->streams[i].open) {
            id = (int)i;
            break;
        }
    if (id < 0) {
        id = (int)s->streams.size();
        s->streams.push_back(S);
    } else {
        s->streams[id] = S;
    }
    s->stats.streams_open += 1;
    *stream_id = id;
    return FT_OK;
}

ft_status ft_server_close_stream(ft_server *s, int sid)
{
    if (!s) return fail(FT_EINVAL, "ft_server_close_stream: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (sid < 0 || sid >= (int)s->streams.size() || !s->streams[sid].open) return fail(FT_EINVAL, "stream %d not open", sid);
    StreamState &S = s->streams[sid];
    if (S.in_flight || S.queued > 0) return fail(FT_EBUSY, "stream %d has requests in flight", sid);
    s->pool->release(S.off, S.bytes);
    free_staging(S);
    S = StreamState();
    s->stats.streams_open -= 1;
    return FT_OK;
}

ft_status ft_server_set_pyramids(ft_server *s, int sid, const ft_pyramid *left, const ft_pyramid *right)
{
    if (!s || !left || !right) return fail(FT_EINVAL, "ft_server_set_pyramids: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (sid < 0 || sid >= (int)s->streams.size() || !s->streams[sid].open) return fail(FT_EINVAL, "stream %d not open", sid);
    StreamState &S = s->streams[sid];
    if (S.desc.camera != FT_CAMERA_PINHOLE) return fail(FT_EINVAL, "stream %d has no pyramids", sid);
    if (S.in_flight) return fail(FT_EBUSY, "stream %d has a request in flight", sid);
    if (s->dry) return FT_OK;
    for (int l = 0; l < S.desc.nlevels; ++l) {
        const int w = S.desc.level_width[l], h = S.desc.level_height[l];
        const ft_pyramid *src[2] = {left, right};
        const size_t dst[2] = {S.o_pyrL[l], S.o_pyrR[l]};
        for (int k = 0; k < 2; ++k) {
            if (!src[k]->data[l] || src[k]->width[l] != w || src[k]->height[l] != h || src[k]->pitch[l] < w)
                return fail(FT_EINVAL, "pyramid level %d does not match the stream", l);
            if (cudaMemcpy2D(S.dev + dst[k], level_pitch(S.desc, l), src[k]->data[l], (size_t)src[k]->pitch[l],
                             (size_t)w, (size_t)h, cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(FT_ECUDA, "pyramid upload failed");
        }
    }
    return FT_OK;
}

ft_status ft_server_set_map(ft_server *s, int sid, const ft_map_view *map)
{
    if (!s || !map) return fail(FT_EINVAL, "ft_server_set_map: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (sid < 0 || sid >= (int)s->streams.size() || !s->streams[sid].open) return fail(FT_EINVAL, "stream %d not open", sid);
    StreamState &S = s->streams[sid];
    if (map->n < 0 || map->n > S.desc.max_map) return fail(FT_EINVAL, "map of %d points exceeds capacity %d", map->n, S.desc.max_map);
    if (S.in_flight) return fail(FT_EBUSY, "stream %d has a request in flight", sid);
    if (!s->dry && map->n > 0) {
        if (!map->pos || !map->nrm || !map->desc) return fail(FT_EINVAL, "map: NULL array");
        const size_t n = (size_t)map->n;
        bool ok = cudaMemcpy(S.dev + S.o_pos, map->pos, 16 * n, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(S.dev + S.o_nrm, map->nrm, 16 * n, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(S.dev + S.o_mdesc, map->desc, 32 * n, cudaMemcpyHostToDevice) == cudaSuccess;
        if (ok) {
            if (map->skip) ok = cudaMemcpy(S.dev + S.o_skip, map->skip, n, cudaMemcpyHostToDevice) == cudaSuccess;
            else ok = cudaMemset(S.dev + S.o_skip, 0, n) == cudaSuccess;
        }
        if (!ok) return fail(FT_ECUDA, "map upload failed");
    }
    S.map_n = map->n;
    return FT_OK;
}

ft_status ft_server_submit(ft_server *s, const ft_request *req)
{
    if (!s || !req) return fail(FT_EINVAL, "ft_server_submit: NULL argument");
    Request r;
    r.tag = req->tag;
    r.sid = req->stream_id;
    r.nl = req->left.n;
    r.nr = req->right.n;
    r.pose = req->pose;
    for (int i = 0; i < 3; ++i) r.O_right[i] = req->O_right[i];
    r.images = req->image_left != nullptr || req->image_right != nullptr;
    char *dst = nullptr, *img = nullptr;
    int W0 = 0, H0 = 0;
    size_t lp0 = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (r.sid < 0 || r.sid >= (int)s->streams.size() || !s->streams[r.sid].open)
            return fail(FT_EINVAL, "stream %d not open", r.sid);
        StreamState &S = s->streams[r.sid];
        if (r.nl < 0 || r.nl > S.desc.max_left || r.nr < 0 || r.nr > S.desc.max_right)
            return fail(FT_EINVAL, "request of %d/%d keypoints exceeds the stream's capacity", r.nl, r.nr);
        if (r.images) {
            if (S.desc.camera != FT_CAMERA_PINHOLE) return fail(FT_EINVAL, "stream %d has no pyramids", r.sid);
            if (!req->image_left || !req->image_right) return fail(FT_EINVAL, "request images: both or neither");
            W0 = S.desc.level_width[0];
            H0 = S.desc.level_height[0];
            if (req->image_pitch < W0) return fail(FT_EINVAL, "image pitch %d below the width %d", req->image_pitch, W0);
            int w[FT_MAX_LEVELS], h[FT_MAX_LEVELS];
            if (ft_pyramid_sizes(W0, H0, &s->params, w, h) != FT_OK) return FT_EINVAL;
            for (int l = 1; l < S.desc.nlevels; ++l)
                if (w[l] != S.desc.level_width[l] || h[l] != S.desc.level_height[l])
                    return fail(FT_EINVAL, "stream level %d is %dx%d; built from level 0 it is %dx%d", l,
                                S.desc.level_width[l], S.desc.level_height[l], w[l], h[l]);
            lp0 = level_pitch(S.desc, 0);
        }
        r.buf = -1;
        for (int b = 0; b < s->depth; ++b)
            if (!S.dyn_used[b]) {
                r.buf = b;
                break;
            }
        if (r.buf < 0) return fail(FT_EBUSY, "stream %d already has %d requests waiting", r.sid, s->depth);
        if (r.images && !s->dry && !S.h_img[r.buf] &&
            cudaMallocHost(&S.h_img[r.buf], 2 * lp0 * (size_t)H0) != cudaSuccess) {
            S.h_img[r.buf] = nullptr;
            return fail(FT_ENOMEM, "pinned image staging for stream %d could not be allocated", r.sid);
        }
        S.dyn_used[r.buf] = 1;
        dst = S.h_dyn[r.buf];
        img = S.h_img[r.buf];
    }
    if (!s->dry) {
        const DynLayout D = dyn_layout(r.nl, r.nr);
        auto cp = [&](size_t off, const void *src, size_t n) {
            if (n) std::memcpy(dst + off, src, n);
        };
        cp(D.lx, req->left.x, 4 * (size_t)r.nl);
        cp(D.ly, req->left.y, 4 * (size_t)r.nl);
        cp(D.loct, req->left.oct, (size_t)r.nl);
        cp(D.ldesc, req->left.desc, 32 * (size_t)r.nl);
        cp(D.rx, req->right.x, 4 * (size_t)r.nr);
        cp(D.ry, req->right.y, 4 * (size_t)r.nr);
        cp(D.roct, req->right.oct, (size_t)r.nr);
        cp(D.rdesc, req->right.desc, 32 * (size_t)r.nr);
        if (req->taken_left) cp(D.tl, req->taken_left, (size_t)r.nl);
        else if (r.nl) std::memset(dst + D.tl, 0, (size_t)r.nl);
        if (req->taken_right) cp(D.tr, req->taken_right, (size_t)r.nr);
        else if (r.nr) std::memset(dst + D.tr, 0, (size_t)r.nr);
        if (r.images) {
            const uint8_t *src[2] = {req->image_left, req->image_right};
            for (int k = 0; k < 2; ++k)
                for (int y = 0; y < H0; ++y)
                    std::memcpy(img + (size_t)k * lp0 * H0 + (size_t)y * lp0,
                                src[k] + (size_t)y * (size_t)req->image_pitch, (size_t)W0);
        }
    }
    r.t_submit = now_us();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->streams[r.sid].queued += 1;
        s->pending.push_back(r);
        s->stats.submitted += 1;
    }
    s->cv.notify_one();
    return FT_OK;
}

int ft_server_poll(ft_server *s, ft_completion *out, int max, int timeout_us)
{
    if (!s || !out || max <= 0) return 0;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->completed.empty() && timeout_us > 0)
        s->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !s->completed.empty(); });
    int n = 0;
    while (n < max && !s->completed.empty()) {
        out[n++] = s->completed.front();
        s->completed.pop_front();
    }
    return n;
}

ft_status ft_server_get_stats(ft_server *s, ft_server_stats *st)
{
    if (!s || !st) return fail(FT_EINVAL, "ft_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->stats;
    st->pool_used = s->pool->used();
    st->pool_capacity = s->pool->capacity();
    st->pending = (uint64_t)s->pending.size();
    st->last_error = s->last_launch_status;
    return FT_OK;
}

}  // extern "C"
