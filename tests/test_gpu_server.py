"""The served loop on the GPU: uneven camera streams (three pinhole
resolutions and fisheye) submit frames continuously; every result that comes
back from the mixed, overlapping batches equals the oracle's result for that
frame alone.  Requests may carry their level-0 images, from which the batch
rebuilds the stream's pyramid on the device."""
import ctypes as C
import time

import numpy as np
import pytest

import oracle as orc
from paper_2509_10757_gb300 import scenes
from tests.gpu_common import assert_fisheye_equal, assert_search_equal, assert_stereo_equal

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2509_10757_gb300 import build
    build.build()
    from paper_2509_10757_gb300 import _lib
    _lib.load()
    return _lib


def test_served_results_equal_solo_results(L):
    from paper_2509_10757_gb300.batch import HostFrame, results_arrays, stream_desc_of
    frames = [scenes.served_stream_frame(1, s) for s in range(8)]
    assert {f.camera for f in frames} == {"pinhole", "fisheye"}
    d = L.ft_server_desc()
    L.ft_server_desc_default(C.byref(d))
    d.hbm_budget, d.n_slots, d.max_batch = 1 << 30, 3, 5
    s = C.c_void_p()
    L.check(L.ft_server_create(C.byref(s), C.byref(d), None), "server")
    try:
        hosts, sids = [], []
        for fr in frames:
            h = HostFrame(fr)
            sid = C.c_int()
            L.check(L.ft_server_open_stream(s, C.byref(stream_desc_of(fr)), C.byref(sid)), "open")
            if fr.camera == "pinhole":
                pl, pr = h.pyramids()
                L.check(L.ft_server_set_pyramids(s, sid.value, C.byref(pl), C.byref(pr)), "pyr")
            L.check(L.ft_server_set_map(s, sid.value, C.byref(h.map_view())), "map")
            hosts.append(h)
            sids.append(sid.value)
        expected = [orc.track_frame(dict(scenes.DEFAULT_PARAMS), fr) for fr in frames]
        buf = (L.ft_completion * 64)()
        got = 0
        n = 0
        for rep in range(3):
            for k, (h, sid) in enumerate(zip(hosts, sids)):
                while L.ft_server_submit(s, C.byref(h.request(sid, 100 * rep + k))) == L.FT_EBUSY:
                    got += check(L, s, buf, frames, expected, sids)
                n += 1
        t0 = time.time()
        while got < n and time.time() - t0 < 60:
            got += check(L, s, buf, frames, expected, sids)
        assert got == n
        stats = L.ft_server_stats()
        L.ft_server_get_stats(s, C.byref(stats))
        assert stats.last_error == 0 and stats.completed == n
        assert stats.batches < n, "requests were batched together"
    finally:
        L.ft_server_destroy(s)


def test_served_requests_carry_images(L):
    # pinhole streams that never upload a pyramid: their requests bring the
    # level-0 images, the server replaces the resident level 0 and the batch
    # builds levels 1.. on the device; results equal the oracle's on the
    # oracle-built pyramids.  A request without images then reuses the levels
    # the previous one built.
    import dataclasses
    from paper_2509_10757_gb300.batch import HostFrame, stream_desc_of
    cands = (scenes.served_stream_frame(3, k) for k in range(40))
    frames = [fr for fr in cands if fr.camera == "pinhole"][:5]
    assert len({fr.pyr_left[0].shape for fr in frames}) > 1
    refs = [dataclasses.replace(fr, pyr_left=orc.build_pyramid(fr.pyr_left[0]),
                                pyr_right=orc.build_pyramid(fr.pyr_right[0])) for fr in frames]
    expected = [orc.track_frame(dict(scenes.DEFAULT_PARAMS), fr) for fr in refs]
    d = L.ft_server_desc()
    L.ft_server_desc_default(C.byref(d))
    d.hbm_budget, d.n_slots, d.max_batch = 1 << 30, 3, 4
    s = C.c_void_p()
    L.check(L.ft_server_create(C.byref(s), C.byref(d), None), "server")
    try:
        hosts, sids = [], []
        for fr in frames:
            h = HostFrame(fr)
            sid = C.c_int()
            L.check(L.ft_server_open_stream(s, C.byref(stream_desc_of(fr)), C.byref(sid)), "open")
            L.check(L.ft_server_set_map(s, sid.value, C.byref(h.map_view())), "map")
            hosts.append(h)
            sids.append(sid.value)
        buf = (L.ft_completion * 64)()
        for rnd, images in enumerate((True, False, True)):
            got, n = 0, 0
            for k, (h, sid) in enumerate(zip(hosts, sids)):
                req = h.request(sid, 100 * rnd + k, images=images)
                while L.ft_server_submit(s, C.byref(req)) == L.FT_EBUSY:
                    got += check(L, s, buf, frames, expected, sids)
                n += 1
            t0 = time.time()
            while got < n and time.time() - t0 < 60:
                got += check(L, s, buf, frames, expected, sids)
            assert got == n, rnd
        stats = L.ft_server_stats()
        L.ft_server_get_stats(s, C.byref(stats))
        assert stats.last_error == 0
    finally:
        L.ft_server_destroy(s)


def check(L, s, buf, frames, expected, sids):
    from paper_2509_10757_gb300.batch import results_arrays
    k = L.ft_server_poll(s, buf, 64, 20000)
    for i in range(k):
        c = buf[i]
        assert c.status == 0
        f = sids.index(c.stream_id)
        fr = frames[f]
        out = results_arrays(c, fr.camera)
        st, se = expected[f]
        where = f"served stream {f} tag {c.tag}: "
        if fr.camera == "pinhole":
            assert_stereo_equal(out, st, where)
            assert_search_equal(out, se, "l", None, where)
        else:
            assert_fisheye_equal(out, st, where)
            assert_search_equal(out, se, "l", "l", where)
            assert_search_equal(out, se, "r", "r", where)
        assert c.t_submit_us <= c.t_start_us <= c.t_done_us
    return k
