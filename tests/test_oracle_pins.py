"""Pins of the CPU oracle against facts fixed outside it: brute force on tiny
inputs, closed forms, invariants, library routines for the general-position
special case, and hand-derived golden values under tests/golden/."""
import os
from fractions import Fraction

import numpy as np
import pytest

import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _f32(x):
    """Round an exact rational to the nearest float32 (ties to even)."""
    x = Fraction(x)
    if x == 0:
        return np.float32(0.0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while a >= Fraction(2) ** (e + 1):
        e += 1
    while a < Fraction(2) ** e:
        e -= 1
    q = a / Fraction(2) ** (e - 23)          # in [2^23, 2^24)
    n = q.numerator // q.denominator
    r = q - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return np.float32(sign * float(Fraction(n) * Fraction(2) ** (e - 23)))


def _interp32(abc_t, u, v):
    """fp32 fma(a, u, fma(b, v, c)) evaluated exactly, then rounded once per fma."""
    a, b, c = (Fraction(float(x)) for x in abc_t)
    inner = _f32(b * v + c)
    return _f32(a * u + Fraction(float(inner)))


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split(":", 1)
        out[k.strip()] = [int(x) for x in v.split()]
    return out


# ---------------------------------------------------------------- census (Sec. III-C)
def _census_brute(img):
    H, W = img.shape
    out = np.zeros((H, W), np.uint32)
    offs = [(dy, dx) for dy in range(-2, 3) for dx in range(-2, 3) if (dy, dx) != (0, 0)]
    for v in range(2, H - 2):
        for u in range(2, W - 2):
            code = 0
            for b, (dy, dx) in enumerate(offs):
                if int(img[v + dy, u + dx]) < int(img[v, u]):
                    code |= 1 << b
            out[v, u] = code
    return out


def test_census_brute_force(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(5):
        img = rng.integers(0, 256, (9, 11), dtype=np.uint8)
        assert np.array_equal(oracle_mod.census(img), _census_brute(img))


def test_census_hand_example(oracle_mod):
    # centre 50; the neighbour at offset (dy, dx) = (-2, -2) is darker -> bit 0;
    # (+2, +2) darker -> bit 23; (0, +1) darker -> bit 12 (row dy=0: dx=-2,-1 are bits 10,11).
    img = np.full((5, 5), 60, np.uint8)
    img[2, 2] = 50
    img[0, 0] = 10
    img[4, 4] = 49
    img[2, 3] = 0
    assert int(oracle_mod.census(img)[2, 2]) == (1 << 0) | (1 << 23) | (1 << 12)


def test_census_invariants(oracle_mod):
    rng = np.random.default_rng(2)
    img = rng.integers(0, 128, (20, 24), dtype=np.uint8)
    c = oracle_mod.census(img)
    # strictly increasing intensity map leaves the codes unchanged
    assert np.array_equal(oracle_mod.census((2 * img.astype(np.int32) + 1).astype(np.uint8)), c)
    pc = np.array([bin(int(x)).count("1") for x in c.ravel()])
    assert pc.max() <= 24
    assert (c[:2] == 0).all() and (c[:, -2:] == 0).all()


def test_omega_brute_force(oracle_mod):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 40, (12, 13), dtype=np.uint8)
    om = oracle_mod.omega(img, t_grad=8)
    H, W = img.shape
    for v in range(H):
        for u in range(W):
            want = 0
            if 2 <= u < W - 2 and 2 <= v < H - 2:
                g = abs(int(img[v, u + 1]) - int(img[v, u - 1])) + abs(int(img[v + 1, u]) - int(img[v - 1, u]))
                want = int(g >= 8)
            assert om[v, u] == want


# ---------------------------------------------------------------- FAST (Sec. III-A)
_CIRCLE = [(0, -3), (1, -3), (2, -2), (3, -1), (3, 0), (3, 1), (2, 2), (1, 3),
           (0, 3), (-1, 3), (-2, 2), (-3, 1), (-3, 0), (-3, -1), (-2, -2), (-1, -3)]


def _fast_brute(img, u, v, t):
    H, W = img.shape
    if not (3 <= u < W - 3 and 3 <= v < H - 3):
        return 0
    p = int(img[v, u])
    ring = np.array([int(img[v + dy, u + dx]) for dx, dy in _CIRCLE])
    bright = ring > p + t
    dark = ring < p - t
    twice_b = np.concatenate([bright, bright])
    twice_d = np.concatenate([dark, dark])
    corner = any(twice_b[s:s + 9].all() or twice_d[s:s + 9].all() for s in range(16))
    if not corner:
        return 0
    return int(max((ring[bright] - p - t).sum(), (p - ring[dark] - t).sum()))


def test_fast_golden_dot(oracle_mod):
    g = _golden("fast_dot.txt")
    img = np.zeros((g["size"][1], g["size"][0]), np.uint8)
    u, v, val = g["dot"]
    img[v, u] = val
    kp = oracle_mod.fast_keypoints(img, t_fast=g["t_fast"][0], K=4)
    assert kp.tolist() == [g["keypoints"]]
    assert oracle_mod.fast_score(img, u, v, g["t_fast"][0]) == g["score"][0]


def test_fast_score_brute_force(oracle_mod):
    rng = np.random.default_rng(4)
    img = (rng.random((24, 30)) * 255).astype(np.uint8)
    img[::3, ::4] = 255
    for v in range(24):
        for u in range(30):
            assert oracle_mod.fast_score(img, u, v, 20) == _fast_brute(img, u, v, 20), (u, v)


def test_fast_bins_brute_force(oracle_mod):
    rng = np.random.default_rng(5)
    img = np.clip(scenes.value_noise(*np.meshgrid(np.arange(96.0), np.arange(70.0)), 77)
                  + rng.normal(0, 6, (70, 96)), 0, 255).astype(np.uint8)
    H, W = img.shape
    S = np.array([[_fast_brute(img, u, v, 12) for u in range(W)] for v in range(H)])
    keep = []
    for v in range(H):
        for u in range(W):
            s = S[v, u]
            if s <= 0:
                continue
            ok = True
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if (dx, dy) == (0, 0) or not (0 <= u + dx < W and 0 <= v + dy < H):
                        continue
                    sn = S[v + dy, u + dx]
                    if sn > s or (sn == s and (v + dy) * W + u + dx < v * W + u):
                        ok = False
            if ok:
                keep.append((12 * u // W + 12 * (10 * v // H), -s, v * W + u, u, v))
    keep.sort()
    want, per = [], {}
    for b, negs, idx, u, v in keep:
        if per.get(b, 0) < 3:
            want.append([u, v])
            per[b] = per.get(b, 0) + 1
    got = oracle_mod.fast_keypoints(img, t_fast=12, K=3)
    assert len(want) > 20
    assert got.tolist() == want


# ---------------------------------------------------------------- epipolar matching
def test_epipolar_integer_shift_closed_form(oracle_mod):
    p = scenes.integer_shift_pair(96, 40, shift=7, seed=3, dmax=32)
    cL, cR = oracle_mod.census(p.left), oracle_mod.census(p.right)
    q = np.array([[u, v] for v in range(2, 38, 5) for u in range(30, 90, 7)], np.int32)
    d = oracle_mod.epipolar_match(cL, cR, q, 32, t_lo=4, margin=2)
    # noise-free shift: cost 0 at d = 7 exactly; accepted wherever unique
    assert (d[d >= 0] == 7).all()
    assert (d == 7).mean() > 0.6


def test_epipolar_brute_force(oracle_mod):
    rng = np.random.default_rng(6)
    H, W = 12, 60
    L = rng.integers(0, 256, (H, W), dtype=np.uint8)
    R = np.roll(L, -5, axis=1)
    R[:, ::7] = rng.integers(0, 256, (H, len(range(0, W, 7))), dtype=np.uint8)
    cL, cR = oracle_mod.census(L), oracle_mod.census(R)
    q = np.array([[u, v] for v in range(2, H - 2) for u in range(2, W - 2)], np.int32)
    for tlo, margin, dmax in ((4, 2, 16), (12, 1, 64), (24, 3, 8)):
        d = oracle_mod.epipolar_match(cL, cR, q, dmax, t_lo=tlo, margin=margin)
        for i, (u, v) in enumerate(q):
            ds = np.arange(0, min(dmax - 1, u - 2) + 1)
            cost = np.array([bin(int(cL[v, u]) ^ int(cR[v, u - k])).count("1") for k in ds])
            best = int(cost.min())
            dstar = int(ds[np.argmax(cost == best)])
            far = cost[np.abs(ds - dstar) >= 2]
            ok = best < tlo and (len(far) == 0 or far.min() >= best + margin)
            assert d[i] == (dstar if ok else -1), (u, v, tlo)


# ---------------------------------------------------------------- Delaunay (Sec. III-A)
def _canon(P):
    P = np.asarray(P, np.int64)
    order = np.lexsort((P[:, 0], P[:, 1]))
    return P[order]


def _orient(a, b, c):
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def _hull_boundary_count(P):
    """Points on the convex hull boundary (vertices and collinear edge points), brute force."""
    n = len(P)
    on = np.zeros(n, bool)
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            s = [_orient(P[i], P[j], P[k]) for k in range(n)]
            if all(x >= 0 for x in s):  # (i, j) supports the hull
                for k in range(n):
                    if s[k] == 0:
                        # on the supporting line and between? collinear points on the hull line
                        on[k] = True
    return int(on.sum())


def _check_valid_delaunay(P, tri):
    """Triangulation covers the hull with positive-area triangles and every
    circumcircle is empty of points strictly inside (exact integers)."""
    P = [tuple(map(int, p)) for p in P]
    area = 0
    for i, j, k in tri:
        o = _orient(P[i], P[j], P[k])
        assert o != 0
        area += abs(o)
        a, b, c = (P[i], P[j], P[k]) if o > 0 else (P[i], P[k], P[j])
        for m, d in enumerate(P):
            if m in (i, j, k):
                continue
            rows = [(x[0] - d[0], x[1] - d[1]) for x in (a, b, c)]
            M = [[dx, dy, dx * dx + dy * dy] for dx, dy in rows]
            det = (M[0][0] * (M[1][1] * M[2][2] - M[2][1] * M[1][2])
                   - M[0][1] * (M[1][0] * M[2][2] - M[2][0] * M[1][2])
                   + M[0][2] * (M[1][0] * M[2][1] - M[2][0] * M[1][1]))
            assert det <= 0, ("point inside circumcircle", (i, j, k), m)
    # hull area (doubled) by a gift-wrapped polygon
    hull = _hull_polygon(P)
    harea = abs(sum(hull[i][0] * hull[(i + 1) % len(hull)][1] - hull[(i + 1) % len(hull)][0] * hull[i][1]
                    for i in range(len(hull))))
    assert area == harea
    used = set(np.asarray(tri).ravel().tolist())
    assert used == set(range(len(P)))


def _hull_polygon(P):
    pts = sorted(set(P))
    if len(pts) < 3:
        return pts

    def half(seq):
        h = []
        for p in seq:
            while len(h) >= 2 and _orient(h[-2], h[-1], p) <= 0:
                h.pop()
            h.append(p)
        return h
    lower, upper = half(pts), half(reversed(pts))
    return lower[:-1] + upper[:-1]


def test_delaunay_golden_square(oracle_mod):
    g = _golden("square_sos.txt")
    P = np.array(g["points"]).reshape(-1, 2)
    assert oracle_mod.delaunay(P).tolist() == np.array(g["triangles"]).reshape(-1, 3).tolist()


def test_delaunay_unit_lattice_closed_form(oracle_mod):
    # every unit square's four corners are the only cocircular set; the
    # smallest index is its (u, v) corner, so each square folds along the
    # diagonal from (u+1, v) to (u, v+1)
    k = 5
    P = _canon([(u, v) for v in range(k) for u in range(k)])
    idx = {tuple(p): i for i, p in enumerate(P.tolist())}
    want = []
    for v in range(k - 1):
        for u in range(k - 1):
            a, b, c, d = idx[(u, v)], idx[(u + 1, v)], idx[(u, v + 1)], idx[(u + 1, v + 1)]
            want.append(sorted((a, b, c)))
            want.append(sorted((b, c, d)))
    assert oracle_mod.delaunay(P).tolist() == sorted(want)


def test_delaunay_general_position_matches_qhull(oracle_mod):
    import scipy.spatial as spatial  # present on every machine this suite runs on: fail, never skip
    rng = np.random.default_rng(7)
    for n in (5, 17, 60, 300):
        P = _canon(np.unique(rng.integers(0, 16000, (n, 2)), axis=0))
        tri = oracle_mod.delaunay(P)
        q = spatial.Delaunay(P.astype(np.float64))
        want = sorted(sorted(map(int, s)) for s in q.simplices)
        assert tri.tolist() == want


def _incircle_exact(a, b, c, d):
    """Sign of the in-circle determinant of d against the CCW triangle abc (exact integers)."""
    rows = [(p[0] - d[0], p[1] - d[1]) for p in (a, b, c)]
    m = [(x, y, x * x + y * y) for x, y in rows]
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


@pytest.mark.parametrize("seed", [41, 42])
def test_delaunay_general_position_brute_force(oracle_mod, seed):
    """Without any library: for points with no three collinear and no four
    cocircular, the Delaunay triangles are exactly the triples whose
    circumcircle holds no other point (enumerated over every triple)."""
    rng = np.random.default_rng(seed)
    while True:
        P = _canon(np.unique(rng.integers(0, 2000, (28, 2)), axis=0))
        n = len(P)
        pts = [tuple(map(int, p)) for p in P]
        trip = [(i, j, k) for i in range(n) for j in range(i + 1, n) for k in range(j + 1, n)]
        if any(_orient(pts[i], pts[j], pts[k]) == 0 for i, j, k in trip):
            continue
        want, degenerate = [], False
        for i, j, k in trip:
            a, b, c = pts[i], pts[j], pts[k]
            if _orient(a, b, c) < 0:
                b, c = c, b
            signs = [_incircle_exact(a, b, c, pts[m]) for m in range(n) if m not in (i, j, k)]
            if 0 in signs:
                degenerate = True
                break
            if all(x < 0 for x in signs):
                want.append([i, j, k])
        if not degenerate:
            break
    assert oracle_mod.delaunay(P).tolist() == want


@pytest.mark.parametrize("seed", [8, 9, 10])
def test_delaunay_degenerate_lattice_valid(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    P = _canon(np.unique(rng.integers(0, 9, (40, 2)), axis=0))
    tri = oracle_mod.delaunay(P)
    _check_valid_delaunay(P, tri.tolist())
    h = _hull_boundary_count(P.tolist())
    assert len(tri) == 2 * len(P) - 2 - h


def test_delaunay_collinear_and_tiny(oracle_mod):
    assert len(oracle_mod.delaunay(np.array([[0, 0], [1, 0]]))) == 0
    assert len(oracle_mod.delaunay(np.array([[0, 0], [3, 0], [7, 0], [9, 0]]))) == 0
    P = _canon([(0, 0), (1, 0), (2, 0), (3, 0), (1, 2)])
    tri = oracle_mod.delaunay(P)
    _check_valid_delaunay(P, tri.tolist())
    assert len(tri) == 3


# ---------------------------------------------------------------- planes + interpolation (Eq. 3)
def test_planes_reproduce_dyadic_plane(oracle_mod):
    rng = np.random.default_rng(11)
    a, b, c = 0.125, -0.0625, 17.5
    P = _canon(np.unique(rng.integers(0, 64, (30, 2)), axis=0))
    D = (a * P[:, 0] + b * P[:, 1] + c).astype(np.float32)
    tri = oracle_mod.delaunay(P)
    abc = oracle_mod.planes(P, D, tri)
    assert (abc == np.float32([a, b, c])).all()
    pidx = oracle_mod.raster(P, tri, 64, 64)
    dmap = oracle_mod.interp_map(pidx, abc)
    uu, vv = np.meshgrid(np.arange(64), np.arange(64))
    assert np.isnan(dmap[pidx < 0]).all()
    assert (dmap[pidx >= 0] == (a * uu + b * vv + c)[pidx >= 0]).all()
    for v in range(64):
        for u in range(64):
            t = pidx[v, u]
            if t >= 0:
                assert _interp32(abc[t], u, v) == np.float32(a * u + b * v + c)


# ---------------------------------------------------------------- raster (Sec. III-B)
def _perturbed_inside(p, tri_pts):
    """Point p + (1/1000, 1/10^6) strictly inside the triangle, exact rationals.
    With coordinates below 100 this shifted point decides every boundary case
    the same way as an infinitesimal shift (1 >> eps, eps >> eps^2)."""
    x = Fraction(p[0]) + Fraction(1, 1000)
    y = Fraction(p[1]) + Fraction(1, 10**6)
    (ax, ay), (bx, by), (cx, cy) = tri_pts
    s = [(bx - ax) * (y - ay) - (by - ay) * (x - ax),
         (cx - bx) * (y - by) - (cy - by) * (x - bx),
         (ax - cx) * (y - cy) - (ay - cy) * (x - cx)]
    return all(t > 0 for t in s) or all(t < 0 for t in s)


@pytest.mark.parametrize("seed", [12, 13])
def test_raster_partition_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    W, H = 40, 30
    P = _canon(np.unique(np.concatenate([rng.integers(0, 40, (25, 2)) * [1, 1],
                                         [[0, 0], [39, 0], [0, 29], [39, 29], [20, 0], [0, 15]]]), axis=0))
    P = P[(P[:, 0] < W) & (P[:, 1] < H)]
    tri = oracle_mod.delaunay(P)
    pidx = oracle_mod.raster(P, tri, W, H)
    for v in range(H):
        for u in range(W):
            hits = [t for t, (i, j, k) in enumerate(tri) if _perturbed_inside((u, v), (P[i], P[j], P[k]))]
            assert len(hits) <= 1
            assert pidx[v, u] == (hits[0] if hits else -1), (u, v)


# ---------------------------------------------------------------- refinement + resampling (Alg. 3, 4)
def test_validate_integer_shift_closed_form(oracle_mod):
    shift, W, H = 6, 80, 48
    p = scenes.integer_shift_pair(W, H, shift=shift, seed=5, dmax=24)
    cL, cR = oracle_mod.census(p.left), oracle_mod.census(p.right)
    om = oracle_mod.omega(p.left)
    # exact support on the plane d = shift
    P = _canon([(u, v) for v in (2, 20, 45) for u in (10, 40, 77)])
    D = np.full(len(P), shift, np.float32)
    tri = oracle_mod.delaunay(P)
    abc = oracle_mod.planes(P, D, tri)
    pidx = oracle_mod.raster(P, tri, W, H)
    Df = np.zeros((H, W), np.float32)
    Cf = np.full((H, W), 8, np.uint8)
    sz = 8
    r = oracle_mod.validate(cL, cR, om, pidx, abc, sz, Df, Cf, t_lo=4, t_hi=8)
    uu, vv = np.meshgrid(np.arange(W), np.arange(H))
    ev = (om == 1) & (pidx >= 0) & (uu - shift >= 2)
    assert ev.sum() > 500
    assert ((r["mask"] & 2) > 0).tolist() == ev.tolist()
    assert (Cf[ev] == 0).all() and (Df[ev] == shift).all()
    assert (Cf[~ev] == 8).all() and (Df[~ev] == 0).all()
    assert not r["cb_w"].any()
    # every cost ties at 0: the first evaluated pixel in raster order wins each cell
    Wc = -(-W // sz)
    for cell in range(len(r["cg_w"])):
        cy, cx = divmod(cell, Wc)
        m = ev[cy * sz:(cy + 1) * sz, cx * sz:(cx + 1) * sz]
        if not m.any():
            assert r["cg_w"][cell] == 0
            continue
        yy, xx = np.argwhere(m)[0]
        assert r["cg_w"][cell] == 1
        assert r["cg_uv"][cell].tolist() == [cx * sz + xx, cy * sz + yy]
        assert r["cg_d"][cell] == shift


def test_validate_tie_breaks_brute_force(oracle_mod):
    rng = np.random.default_rng(14)
    W, H, sz = 37, 29, 4
    L = rng.integers(0, 256, (H, W), dtype=np.uint8)
    R = rng.integers(0, 256, (H, W), dtype=np.uint8)
    cL, cR = oracle_mod.census(L), oracle_mod.census(R)
    om = oracle_mod.omega(L, t_grad=0)
    P = _canon([(0, 0), (36, 0), (0, 28), (36, 28), (18, 14), (9, 20)])
    D = np.array([3, 0, 5, 1, 2, 4], np.float32)[:len(P)]
    tri = oracle_mod.delaunay(P)
    abc = oracle_mod.planes(P, D, tri)
    pidx = oracle_mod.raster(P, tri, W, H)
    Df = np.zeros((H, W), np.float32)
    Cf = np.full((H, W), 14, np.uint8)
    t_lo, t_hi = 11, 13
    r = oracle_mod.validate(cL, cR, om, pidx, abc, sz, Df, Cf, t_lo=t_lo, t_hi=t_hi)
    # brute force: recompute each evaluated pixel's cost, then per cell the
    # lexicographic minimum of (cost, v, u) below t_lo and of (-cost, v, u) above t_hi
    Wc, Hc = -(-W // sz), -(-H // sz)
    best_g, best_b = {}, {}
    for v in range(H):
        for u in range(W):
            t = pidx[v, u]
            if not om[v, u] or t < 0:
                continue
            d = _interp32(abc[t], u, v)
            k = int(np.rint(d))
            if not (2 <= u - k <= W - 3):
                continue
            cost = bin(int(cL[v, u]) ^ int(cR[v, u - k])).count("1")
            cell = (v // sz) * Wc + u // sz
            if cost < t_lo:
                best_g[cell] = min(best_g.get(cell, (99,)), (cost, v, u))
            if cost > t_hi:
                best_b[cell] = min(best_b.get(cell, (99,)), (-cost, v, u))
    assert len(best_g) > 5 and len(best_b) > 5
    for cell in range(Wc * Hc):
        assert r["cg_w"][cell] == (cell in best_g)
        if cell in best_g:
            assert r["cg_uv"][cell].tolist() == [best_g[cell][2], best_g[cell][1]]
            assert r["cg_cost"][cell] == best_g[cell][0]
        assert r["cb_w"][cell] == (cell in best_b)
        if cell in best_b:
            assert r["cb_uv"][cell].tolist() == [best_b[cell][2], best_b[cell][1]]


def test_run_integer_shift_end_to_end(oracle_mod):
    shift = 5
    p = scenes.integer_shift_pair(160, 96, shift=shift, seed=9, dmax=16, texture="iid", flat_left=shift + 5)
    r = oracle_mod.run(p.left, p.right, 16, 3, 16, t_lo=4, t_hi=8, t_fast=10, kp_per_bin=2)
    assert len(r["support"][0]) >= 3
    # every support point of every iteration sits on the true plane
    for S in r["support"]:
        assert (S[:, 2] == shift).all()
    assert len(r["support"][2]) > len(r["support"][1]) > len(r["support"][0])
    got = r["C_f"] < 8
    assert got.sum() > 2000
    assert (r["D_f"][got] == shift).all() and (r["C_f"][got] == 0).all()


def test_accuracy_sanity_band(oracle_mod):
    """Not a pin: the semi-dense output is mostly right on a synthetic polygon scene."""
    p = scenes.config_pairs("vga_polygons")[0]
    r = oracle_mod.run(p.left, p.right, p.dmax, p.iters, p.cell)
    valid = r["C_f"] < 8
    m = valid & ~p.gt_occ
    acc = (np.abs(r["D_f"] - p.gt_disp)[m] < 3).mean()
    assert valid.mean() > 0.2 and acc > 0.6


def test_omega_dense_is_the_interior(oracle_mod):
    """t_grad = 0 (the dense variant): Omega_I is every pixel at least 2 pixels
    from the border, and nothing else, whatever the image (the gradient sum is
    never negative)."""
    rng = np.random.default_rng(21)
    for W, H in [(5, 5), (9, 7), (40, 23)]:
        img = rng.integers(0, 256, (H, W), dtype=np.uint8)
        om = oracle_mod.omega(img, t_grad=0)
        want = np.zeros((H, W), bool)
        want[2:H - 2, 2:W - 2] = True
        assert np.array_equal(om.astype(bool), want)
