"""The allocation-free free-flight entry point against the regular one.

ugp_sample_free_flight_noalloc serves callers that cannot allocate device memory: its scratch
lives in a fixed device array inside the library, without per-ray slot lists, so every bracketed
ray is finished by a warp that rebuilds its intervals by traversal, where the regular entry
point finishes most rays on 16 lanes from the slot list.  Through the C ABI it must give the
same samples bit for bit (the finish sums in fixed point, so neither the collection path nor
the lane count may change a result), on two calls in a row (the second reuses the array the
first left behind) and on a third with exactly as many rays as the array holds (the last column
of its layout in use), and reject more rays than the array holds.  This file runs last so a
failure here leaves every other test already run.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2406_09733_gb300 import scenes

pytestmark = pytest.mark.gpu

MAX_RAYS = 65536


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_09733_gb300 import build, ugp
    build.build()
    L = ugp.lib()
    vp = C.c_void_p
    L.ugp_sample_free_flight_noalloc.restype = C.c_int
    L.ugp_sample_free_flight_noalloc.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    return torch, ugp, L


def _noalloc(torch, ugp, L, bvh, r, u, u2, excl=None):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    o, d, t0, t1, U, U2 = dev(r.o), dev(r.d), dev(r.t0), dev(r.t1), dev(u), dev(u2)
    ex = None if excl is None else dev(excl)
    n = r.n
    prim = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    tu = torch.zeros(n, dtype=torch.float32, device="cuda")
    tsp = torch.zeros(n, dtype=torch.float32, device="cuda")
    st = torch.zeros(n, dtype=torch.uint8, device="cuda")
    p = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    status = L.ugp_sample_free_flight_noalloc(C.c_void_p(bvh.handle), n, p(o), p(d), p(t0), p(t1), p(U), p(U2),
                                              p(ex), p(prim), p(tu), p(tsp), p(st),
                                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return status, prim.cpu().numpy(), tu.cpu().numpy(), tsp.cpu().numpy(), st.cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice(env):
    torch, ugp, L = env
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    # dense aggregates, so the scratch queue is really used
    s = scenes.room_scene(100_000, seed=3, n_clusters=30)
    bvh = ugp.build_bvh(dev(s.mean), dev(s.quat), dev(s.scale), dev(s.magnitude))
    # two calls in a row, then one that fills the fixed array exactly
    for seed, n in ((5, 40000), (6, 40017), (7, MAX_RAYS)):
        r = scenes.random_rays(n, seed=seed, centre=(0.5, 0.5, 0.5), radius=1.2)
        u, u2 = scenes.uniforms24(seed + 10, r.n), scenes.uniforms24(seed + 20, r.n)
        status, prim, tu, tsp, st = _noalloc(torch, ugp, L, bvh, r, u, u2)
        assert status == 0, L.ugp_last_error()
        ref_p, ref_tu, ref_tsp, ref_st = (x.cpu().numpy() for x in ugp.sample_free_flight(
            bvh, dev(r.o), dev(r.d), dev(r.t0), dev(r.t1), dev(u), dev(u2)))
        assert np.array_equal(st, ref_st) and st.max() == 0
        assert np.array_equal(prim, ref_p)
        assert (prim >= 0).mean() > 0.3
        assert np.array_equal(tu, ref_tu)
        assert np.array_equal(tsp, ref_tsp)


def test_noalloc_rejects_more_rays_than_its_array(env):
    torch, ugp, L = env
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    s = scenes.tiny_scene(n=100)
    bvh = ugp.build_bvh(dev(s.mean), dev(s.quat), dev(s.scale), dev(s.magnitude))
    r = scenes.random_rays(MAX_RAYS + 1, seed=9)
    u = scenes.uniforms24(9, r.n)
    status, *_ = _noalloc(torch, ugp, L, bvh, r, u, u)
    assert status == 1 and b"exceed" in L.ugp_last_error()
