"""The device re-tessellation (insertion into the previous mesh + Lawson flips
with the exact, symbolically perturbed predicates) against the host
triangulation and the oracle's own (gift wrapping): identical triangle lists
on random sets, lattices (every cell cocircular), collinear rows, and the
support sets S_1 -> S_2 -> S_3 of both scene generators."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1511_00758_gb300 as S  # noqa: E402


def _canon(P):
    P = np.unique(np.asarray(P, np.int64).reshape(-1, 2), axis=0)
    return np.ascontiguousarray(P[np.lexsort((P[:, 0], P[:, 1]))], dtype=np.int32)


def _host(P):
    tri = np.zeros((2 * len(P) + 8, 3), np.int32)
    T = S.delaunay(P, len(P), tri, len(tri))
    return tri[:T].copy()


def _insert(P, tri, new, W, H):
    new = np.ascontiguousarray(np.asarray(new, np.int32).reshape(-1, 2))
    out = np.zeros((2 * (len(P) + len(new)) + 8, 3), np.int32)
    T = S.delaunay_insert(P, len(P), np.ascontiguousarray(tri), len(tri), new, len(new), W, H, out, len(out))
    return out[:T].copy()


def _covered(oracle_mod, P, tri, W, H, cand):
    """The candidates the old mesh's raster covers (the pixels a pass evaluates)."""
    pidx = oracle_mod.raster(P, tri, W, H)
    cand = np.asarray(cand).reshape(-1, 2)
    return cand[pidx[cand[:, 1], cand[:, 0]] >= 0]


def _check(oracle_mod, P, new, W, H, with_oracle=True):
    tri = _host(P)
    got = _insert(P, tri, new, W, H)
    U = _canon(np.concatenate([P, np.asarray(new, np.int32).reshape(-1, 2)]))
    want = _host(U)
    assert got.shape == want.shape and np.array_equal(got, want)
    if with_oracle:
        assert np.array_equal(got, oracle_mod.delaunay(U))
    return got


def test_insert_random_points(oracle_mod):
    rng = np.random.default_rng(51)
    W, H = 320, 240
    corners = [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1)]
    P = _canon(np.concatenate([rng.integers(0, [W, H], (150, 2)), corners]))
    tri = _host(P)
    new = _covered(oracle_mod, P, tri, W, H, rng.integers(0, [W, H], (600, 2)))
    assert len(new) > 500
    _check(oracle_mod, P, new, W, H)


def test_insert_lattice_cocircular(oracle_mod):
    """Coarse lattice into a fine one: every new point is cocircular with its
    neighbours and many lie on old edges (edge splits, hull splits)."""
    W, H = 97, 65
    P = _canon([(u, v) for v in range(0, H, 16) for u in range(0, W, 16)])
    tri = _host(P)
    new = _covered(oracle_mod, P, tri, W, H, [(u, v) for v in range(0, H, 4) for u in range(0, W, 4)])
    _check(oracle_mod, P, new, W, H)


def test_insert_collinear_rows_and_hull_edges(oracle_mod):
    W, H = 120, 60
    P = _canon([(u, v) for v in (5, 30, 55) for u in (3, 40, 77, 114)])
    tri = _host(P)
    cand = [(u, v) for v in (5, 17, 30, 42, 55) for u in range(3, 115, 3)] + [(3, v) for v in range(5, 56)]
    new = _covered(oracle_mod, P, tri, W, H, cand)
    _check(oracle_mod, P, new, W, H)


def test_insert_nothing_and_only_existing_points(oracle_mod):
    rng = np.random.default_rng(52)
    W, H = 64, 48
    P = _canon(np.concatenate([rng.integers(0, [W, H], (40, 2)), [(0, 0), (63, 0), (0, 47), (63, 47)]]))
    tri = _host(P)
    assert np.array_equal(_insert(P, tri, np.zeros((0, 2), np.int32), W, H), tri)
    assert np.array_equal(_insert(P, tri, P[::3], W, H), tri)


def test_insert_rejects_a_point_outside_the_mesh():
    W, H = 64, 48
    P = _canon([(10, 10), (50, 10), (10, 40), (50, 40)])
    tri = _host(P)
    with pytest.raises(S.StereoError) as e:
        _insert(P, tri, [(60, 45)], W, H)
    assert e.value.code == -1


@pytest.mark.parametrize("kind", ["vga_polygons", "driving_1242x375"])
def test_insert_scene_support_sets(oracle_mod, kind):
    """S_1 -> S_2 -> S_3 of the oracle's own run: each set's triangulation by
    insertion into the previous one equals the host's and the oracle's."""
    p = scenes.config_pairs(kind)[0]
    iters = max(p.iters, 3)
    r = oracle_mod.run(p.left, p.right, p.dmax, iters, p.cell)
    H, W = p.left.shape
    for it in range(1, iters):
        P = _canon(r["support"][it - 1][:, :2])
        Q = _canon(r["support"][it][:, :2])
        old = {tuple(x) for x in P.tolist()}
        new = np.array([x for x in Q.tolist() if tuple(x) not in old], np.int32).reshape(-1, 2)
        assert len(new) > 0
        got = _check(oracle_mod, P, new, W, H, with_oracle=False)
        assert len(got) == int(r["n_tri"][it])
