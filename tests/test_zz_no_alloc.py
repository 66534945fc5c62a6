"""stereo_raster_noalloc against stereo_raster.

The allocation-free raster serves callers that cannot allocate device memory
where they run the raster (fixed real-time memory plans, allocators owned by
another component, captured work); it keeps its work lists in one fixed
device array instead of caller scratch.  Two calls in a row on different
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
