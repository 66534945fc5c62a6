"""stereo_raster_noalloc against stereo_raster.

The allocation-free raster serves callers that cannot allocate device memory
where they run the raster (a real-time loop whose memory is all allocated up
front, or code running while another component owns the device allocator);
it keeps its work lists in one fixed device array instead of caller scratch.
Two calls in a row on different
meshes must each give exactly the plane-index map and D_it that the
scratch-taking entry point gives, so nothing from the first call leaks into
the second through the shared array.  This file is collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1511_00758_gb300 as S  # noqa: E402

DEV = "cuda:0"


def _mesh(seed, n, W, H):
    rng = np.random.default_rng(seed)
    P = np.unique(np.stack([rng.integers(0, W, n), rng.integers(0, H, n)], 1), axis=0)
    P = np.ascontiguousarray(P[np.lexsort((P[:, 0], P[:, 1]))], dtype=np.int32)
    D = rng.uniform(0, 100, len(P)).astype(np.float32)
    tri = np.zeros((2 * len(P) + 8, 3), np.int32)
    T = S.delaunay(P, len(P), tri, len(tri))
    abc = np.zeros((T, 3), np.float32)
    S.planes(P, D, tri[:T], T, abc)
    tuv = np.ascontiguousarray(P[tri[:T]].reshape(-1, 6), dtype=np.int32)
    return tuv, abc, T


def _run(fn_noalloc, tuv, abc, T, W, H):
    t_uv = torch.from_numpy(tuv).to(DEV)
    t_abc = torch.from_numpy(abc).to(DEV)
    pidx = torch.empty((H, W), dtype=torch.int32, device=DEV)
    dit = torch.empty((H, W), dtype=torch.float32, device=DEV)
    if fn_noalloc:
        S.raster_noalloc(t_uv, t_abc, T, W, H, pidx, dit)
    else:
        nbytes = S.raster_scratch_bytes(T)
        scratch = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=DEV)
        S.raster(t_uv, t_abc, T, W, H, pidx, dit, scratch, nbytes)
    torch.cuda.synchronize()
    return pidx.cpu().numpy(), dit.cpu().numpy()


def test_noalloc_raster_matches_scratch_raster_twice():
    S.load()
    cases = [(_mesh(21, 9000, 1242, 375), 1242, 375), (_mesh(22, 300, 640, 480), 640, 480)]
    for (tuv, abc, T), W, H in cases:  # two calls in a row, different meshes
        want_p, want_d = _run(False, tuv, abc, T, W, H)
        got_p, got_d = _run(True, tuv, abc, T, W, H)
        assert np.array_equal(got_p, want_p)
        assert np.array_equal(np.isnan(got_d), np.isnan(want_d))
        ok = ~np.isnan(want_d)
        assert np.array_equal(got_d[ok].view(np.uint32), want_d[ok].view(np.uint32))
        assert (got_p >= 0).mean() > 0.5


def test_noalloc_rejects_too_many_triangles():
    S.load()
    pidx = torch.empty((16, 16), dtype=torch.int32, device=DEV)
    with pytest.raises(S.StereoError) as e:
        S.raster_noalloc(pidx, None, 262144, 16, 16, pidx, None)
    assert e.value.code == -9


def test_noalloc_near_the_triangle_cap():
    """A mesh just under the 262143-triangle limit uses the last entries of the
    fixed array (the block offsets after both lists) and still matches."""
    S.load()
    W, H = 1242, 375
    rng = np.random.default_rng(23)
    m = 131100
    while True:  # distinct pixels: T = 2m - 2 - (hull vertices), trimmed until it fits
        idx = np.sort(rng.choice(W * H, size=m, replace=False))
        P = np.ascontiguousarray(np.stack([idx % W, idx // W], 1), dtype=np.int32)  # (v, u) order
        tri = np.zeros((2 * m + 8, 3), np.int32)
        T = S.delaunay(P, m, tri, len(tri))
        if T <= 262143:
            break
        m -= (T - 262143 + 1) // 2 + 1
    assert 262143 - 1000 < T <= 262143
    D = rng.uniform(0, 100, m).astype(np.float32)
    abc = np.zeros((T, 3), np.float32)
    S.planes(P, D, tri[:T], T, abc)
    tuv = np.ascontiguousarray(P[tri[:T]].reshape(-1, 6), dtype=np.int32)
    want_p, want_d = _run(False, tuv, abc, T, W, H)
    got_p, got_d = _run(True, tuv, abc, T, W, H)
    assert np.array_equal(got_p, want_p)
    ok = ~np.isnan(want_d)
    assert np.array_equal(np.isnan(got_d), ~ok)
    assert np.array_equal(got_d[ok].view(np.uint32), want_d[ok].view(np.uint32))


def test_noalloc_leaves_free_device_memory_unchanged():
    """After one warm call (module loading may take device memory once), a call
    leaves the device's free memory exactly as it was: nothing is allocated."""
    S.load()
    W, H = 640, 480
    tuv, abc, T = _mesh(24, 2000, W, H)
    t_uv = torch.from_numpy(tuv).to(DEV)
    t_abc = torch.from_numpy(abc).to(DEV)
    pidx = torch.empty((H, W), dtype=torch.int32, device=DEV)
    dit = torch.empty((H, W), dtype=torch.float32, device=DEV)
    S.raster_noalloc(t_uv, t_abc, T, W, H, pidx, dit)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        S.raster_noalloc(t_uv, t_abc, T, W, H, pidx, dit)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
