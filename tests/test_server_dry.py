"""Scheduling and admission logic of the served loop, on the CPU: a dry-run
server runs the real scheduler and HBM-budget accounting with fake batch
completions instead of GPU work (the failure and timing are made on the
host).  Checks: admission refuses a stream the budget cannot hold and
accepts it once another stream closes; a stream's requests complete in
submit order and never overlap; batches never exceed max_batch and hold at
most one request per stream; a stream holds as many requests as the queue
depth (two by default) and refuses one more; every request completes;
requests with level-0
images are checked at submit (pinhole streams only, both images, a pitch of
at least the width, stream levels of the sizes the device would build)."""
import ctypes as C
import time

import pytest

from paper_2509_10757_gb300 import scenes


@pytest.fixture(scope="module")
def L():
    from paper_2509_10757_gb300 import build
    build.build()
    from paper_2509_10757_gb300 import _lib
    _lib.load()
    return _lib


def make_server(L, budget=64 << 20, slots=2, max_batch=4, latency_us=300.0, depth=0):
    d = L.ft_server_desc()
    L.ft_server_desc_default(C.byref(d))
    d.hbm_budget, d.n_slots, d.max_batch, d.queue_depth = budget, slots, max_batch, depth
    d.dry_run, d.dry_run_latency_us = 1, latency_us
    s = C.c_void_p()
    L.check(L.ft_server_create(C.byref(s), C.byref(d), None), "server")
    return s


@pytest.fixture(scope="module")
def frames():
    return [scenes.pinhole_frame(s, W=320, H=240, n_left=200, n_map=300) for s in range(3)] + \
           [scenes.fisheye_frame(5, n_left=200, n_map=300)]


def open_stream(L, s, fr):
    from paper_2509_10757_gb300.batch import stream_desc_of
    sid = C.c_int(-1)
    st = L.ft_server_open_stream(s, C.byref(stream_desc_of(fr)), C.byref(sid))
    return st, sid.value


def drain(L, s, n, timeout=10.0):
    out = []
    buf = (L.ft_completion * 64)()
    t0 = time.time()
    while len(out) < n and time.time() - t0 < timeout:
        k = L.ft_server_poll(s, buf, 64, 20000)
        out += [(buf[i].tag, buf[i].stream_id, buf[i].t_submit_us, buf[i].t_start_us, buf[i].t_done_us)
                for i in range(k)]
    return out


def test_budget_admission_and_release(L, frames):
    from paper_2509_10757_gb300.batch import stream_desc_of
    # measure one stream's block by filling a small pool
    s = make_server(L, budget=3 << 20)
    try:
        ids = []
        while True:
            st, sid = open_stream(L, s, frames[0])
            if st != L.FT_OK:
                assert st == L.FT_EBUSY and "HBM budget" in L.last_error()
                break
            ids.append(sid)
            assert len(ids) < 100
        assert len(ids) >= 1
        stats = L.ft_server_stats()
        L.ft_server_get_stats(s, C.byref(stats))
        assert stats.streams_open == len(ids) and stats.pool_used <= stats.pool_capacity
        L.check(L.ft_server_close_stream(s, ids[-1]), "close")
        st, sid = open_stream(L, s, frames[0])
        assert st == L.FT_OK and sid == ids[-1]
    finally:
        L.ft_server_destroy(s)


def test_order_overlap_and_batch_limits(L, frames):
    from paper_2509_10757_gb300.batch import HostFrame
    s = make_server(L, max_batch=2, slots=2, latency_us=2000.0)
    try:
        hf = [HostFrame(f) for f in frames]
        sids = [open_stream(L, s, f)[1] for f in frames]
        tag = 0
        expected = {}
        for rep in range(2):
            for sid, h in zip(sids, hf):
                L.check(L.ft_server_submit(s, C.byref(h.request(sid, tag))), "submit")
                expected.setdefault(sid, []).append(tag)
                tag += 1
        # a third waiting request of one stream is refused
        r = L.ft_server_submit(s, C.byref(hf[0].request(sids[0], 999)))
        assert r == L.FT_EBUSY
        # a stream with requests queued cannot close
        assert L.ft_server_close_stream(s, sids[1]) == L.FT_EBUSY
        done = drain(L, s, tag)
        assert len(done) == tag
        for sid in sids:
            mine = [d for d in done if d[1] == sid]
            assert [d[0] for d in mine] == expected[sid], "a stream's requests complete in order"
            for a, b in zip(mine, mine[1:]):
                assert b[3] >= a[4] - 1e-3, "a stream's requests never overlap"
        stats = L.ft_server_stats()
        L.ft_server_get_stats(s, C.byref(stats))
        assert stats.completed == stats.submitted == tag
        assert stats.frames_launched == tag
        assert stats.batches >= (tag + 1) // 2, "no batch holds more than max_batch"
        # batches of the same slot run one after another; two slots overlap
        starts = sorted(d[3] for d in done)
        assert len(set(starts)) >= 2
    finally:
        L.ft_server_destroy(s)


def test_every_request_completes_under_load(L, frames):
    from paper_2509_10757_gb300.batch import HostFrame
    s = make_server(L, max_batch=8, slots=3, latency_us=200.0)
    try:
        hf = HostFrame(frames[1])
        sids = [open_stream(L, s, frames[1])[1] for _ in range(12)]
        n = 0
        for rep in range(20):
            for sid in sids:
                while L.ft_server_submit(s, C.byref(hf.request(sid, n))) == L.FT_EBUSY:
                    time.sleep(0.0005)
                n += 1
        done = drain(L, s, n, timeout=30)
        assert len(done) == n and len({d[0] for d in done}) == n
        lat = sorted(d[4] - d[2] for d in done)
        assert lat[0] >= 200.0 * 0.9
    finally:
        L.ft_server_destroy(s)


def test_request_images_are_checked_at_submit(L, frames):
    import numpy as np

    from paper_2509_10757_gb300.batch import HostFrame, stream_desc_of
    s = make_server(L)
    try:
        pin, fish = frames[0], frames[3]
        st, sp = open_stream(L, s, pin)
        assert st == L.FT_OK
        st, sf = open_stream(L, s, fish)
        assert st == L.FT_OK
        bad = stream_desc_of(pin)
        bad.level_width[3] += 1                      # not the size built from level 0
        sb = C.c_int(-1)
        assert L.ft_server_open_stream(s, C.byref(bad), C.byref(sb)) == L.FT_OK
        hp, hf = HostFrame(pin), HostFrame(fish)
        img = np.zeros_like(pin.pyr_left[0])
        r = hp.request(sp, 1, images=True)
        r.image_right = None                         # one image only
        assert L.ft_server_submit(s, C.byref(r)) == L.FT_EINVAL
        r = hp.request(sp, 2, images=True)
        r.image_pitch = img.shape[1] - 1             # pitch below the width
        assert L.ft_server_submit(s, C.byref(r)) == L.FT_EINVAL
        r = hf.request(sf, 3)
        r.image_left = r.image_right = img.ctypes.data
        r.image_pitch = img.shape[1]                 # a fisheye stream has no pyramid
        assert L.ft_server_submit(s, C.byref(r)) == L.FT_EINVAL
        assert L.ft_server_submit(s, C.byref(hp.request(sb.value, 4, images=True))) == L.FT_EINVAL
        assert L.ft_server_submit(s, C.byref(hp.request(sb.value, 5))) == L.FT_OK   # no images: accepted
        assert L.ft_server_submit(s, C.byref(hp.request(sp, 6, images=True))) == L.FT_OK
        assert sorted(t for t, *_ in drain(L, s, 2)) == [5, 6]
    finally:
        L.ft_server_destroy(s)


def test_queue_depth_bounds_the_waiting_requests(L, frames):
    from paper_2509_10757_gb300.batch import HostFrame
    d = L.ft_server_desc()
    L.ft_server_desc_default(C.byref(d))
    d.dry_run = 1
    for bad in (-1, 9):
        d.queue_depth = bad
        s = C.c_void_p()
        assert L.ft_server_create(C.byref(s), C.byref(d), None) == L.FT_EINVAL
        assert not s.value
    s = make_server(L, latency_us=3000.0, depth=4)
    try:
        hf = HostFrame(frames[0])
        sid = open_stream(L, s, frames[0])[1]
        for tag in range(4):
            L.check(L.ft_server_submit(s, C.byref(hf.request(sid, tag))), "submit")
        assert L.ft_server_submit(s, C.byref(hf.request(sid, 99))) == L.FT_EBUSY
        assert "4 requests waiting" in L.last_error()
        done = drain(L, s, 4)
        assert [x[0] for x in done] == [0, 1, 2, 3]
    finally:
        L.ft_server_destroy(s)
