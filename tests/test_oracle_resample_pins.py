"""Pins of the oracle's SupportResampling (Alg. 4): the C_b -> epipolar-match
branch and the precedence of the support-set merge, on hand-built cell records
with a hand-derived result (tests/golden/resample_cells.txt), and a closed-form
scene in which a wrong prior sends cells through the match branch and the
matches recover the true integer shift."""
import os

import numpy as np

import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_case(name):
    case = dict(shift={}, reject=[], S=[], cg=[], cb=[], expect=[])
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = (x.strip() for x in line.split(":", 1))
        f = v.split()
        if k == "dims":
            case["W"], case["H"], case["sz"], case["dmax"], case["t_lo"], case["margin"] = map(int, f)
        elif k == "shift":
            case["shift"][int(f[0])] = int(f[1])
        elif k == "reject_row":
            case["reject"].append(int(f[0]))
        elif k in ("S", "expect"):
            case[k].append((int(f[0]), int(f[1]), float(f[2])))
        elif k == "cg":
            case["cg"].append((int(f[0]), int(f[1]), int(f[2]), float(f[3])))
        elif k == "cb":
            case["cb"].append((int(f[0]), int(f[1]), int(f[2])))
    return case


def _distant_codes(rng, n, min_dist):
    """n 24-bit codes, every two of which differ in at least min_dist bits."""
    out = []
    while len(out) < n:
        c = int(rng.integers(0, 1 << 24))
        if all(bin(c ^ o).count("1") >= min_dist for o in out):
            out.append(c)
    return out


def _census_rows(case, seed=3):
    W, H = case["W"], case["H"]
    rng = np.random.default_rng(seed)
    cL = np.zeros((H, W), np.uint32)
    cR = np.zeros((H, W), np.uint32)
    for v in range(H):
        if v in case["reject"]:
            cL[v, :] = 0xFFFFFF
            cR[v, :] = 0
            continue
        s = case["shift"].get(v, 0)
        G = _distant_codes(rng, W + s, 6)
        cL[v, :] = G[:W]
        cR[v, :] = G[s:s + W]  # cR(x) = G(x + s)
    return cL, cR


def _cells(case):
    W, H, sz = case["W"], case["H"], case["sz"]
    nc = (-(-W // sz)) * (-(-H // sz))
    r = dict(cg_uv=np.zeros((nc, 2), np.int32), cg_d=np.zeros(nc, np.float32), cg_w=np.zeros(nc, np.uint8),
             cb_uv=np.zeros((nc, 2), np.int32), cb_w=np.zeros(nc, np.uint8))
    for c, u, v, d in case["cg"]:
        r["cg_uv"][c] = (u, v)
        r["cg_d"][c] = d
        r["cg_w"][c] = 1
    for c, u, v in case["cb"]:
        r["cb_uv"][c] = (u, v)
        r["cb_w"][c] = 1
    return r


def test_golden_codes_have_the_stated_distances():
    """The construction the golden derivation relies on: on a shifted row the
    true shift costs 0 and every other column at least 6 bits."""
    case = _read_case("resample_cells.txt")
    cL, cR = _census_rows(case)
    for v, s in case["shift"].items():
        for u in range(s, case["W"]):
            costs = [bin(int(cL[v, u]) ^ int(cR[v, u - d])).count("1") for d in range(0, u + 1)]
            assert costs[s] == 0
            assert all(c >= 6 for d, c in enumerate(costs) if d != s)


def test_resample_hand_built_records(oracle_mod):
    """Each branch of the merge: a C_g pick on a pixel of S_it is dropped, a
    C_g pick is taken before an X match on the same pixel, an accepted X query
    adds (u, v, d*), a rejected one adds nothing, an X match on a pixel of S_it
    is dropped, and the result is in (v, u) order."""
    case = _read_case("resample_cells.txt")
    cL, cR = _census_rows(case)
    got = oracle_mod.resample(cL, cR, case["sz"], _cells(case), np.array(case["S"], np.float64),
                              case["dmax"], t_lo=case["t_lo"], margin=case["margin"])
    want = np.array(case["expect"], np.float64)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


def test_resample_single_branches(oracle_mod):
    """The same records one at a time, so each reading fails on its own."""
    case = _read_case("resample_cells.txt")
    cL, cR = _census_rows(case)
    S0 = np.array(case["S"], np.float64)

    def one(cg=(), cb=()):
        c = dict(case, cg=list(cg), cb=list(cb))
        return oracle_mod.resample(cL, cR, case["sz"], _cells(c), S0, case["dmax"],
                                   t_lo=case["t_lo"], margin=case["margin"])

    def with_pts(*pts):
        return np.array(sorted(list(map(tuple, S0)) + list(pts), key=lambda p: (p[1], p[0])), np.float64)

    # a C_g pick on an existing support point leaves S_it as it was
    assert np.array_equal(one(cg=[(1, 5, 2, 2.5)]), S0)
    # an accepted X query adds its match; one out of the search range, on a
    # row without a match or without a census code adds nothing
    assert np.array_equal(one(cb=[(1, 7, 2)]), with_pts((7, 2, 3.0)))
    assert np.array_equal(one(cb=[(13, 4, 8)]), with_pts((4, 8, 1.0)))
    assert np.array_equal(one(cb=[(0, 3, 2)]), S0)
    assert np.array_equal(one(cb=[(7, 6, 5)]), S0)
    assert np.array_equal(one(cb=[(17, 22, 8)]), S0)
    # an X match on an existing support point is dropped
    assert np.array_equal(one(cb=[(3, 14, 2)]), S0)
    # C_g before X on the same pixel, whichever cell comes first
    assert np.array_equal(one(cg=[(8, 10, 6, 3.5)], cb=[(9, 10, 6)]), with_pts((10, 6, 3.5)))
    assert np.array_equal(one(cg=[(9, 10, 6, 3.5)], cb=[(8, 10, 6)]), with_pts((10, 6, 3.5)))
    # alone, that X query is accepted with the row's shift
    assert np.array_equal(one(cb=[(9, 10, 6)]), with_pts((10, 6, 4.0)))


def _canon(P):
    return np.array(sorted(P, key=lambda p: (p[1], p[0])), np.int32)


def test_resample_match_branch_recovers_the_shift(oracle_mod):
    """Closed form: on an exact integer-shift pair (no noise, i.i.d. texture), a
    mesh whose support points in one region carry a wrong disparity gives that
    region costs above t_hi, so its cells go through the epipolar match, and
    the match of every such pixel in range is the true shift."""
    shift, W, H, sz, dmax = 5, 96, 48, 8, 24
    p = scenes.integer_shift_pair(W, H, shift=shift, seed=31, dmax=dmax, texture="iid")
    cL, cR = oracle_mod.census(p.left), oracle_mod.census(p.right)
    om = oracle_mod.omega(p.left, t_grad=0)
    P = _canon([(u, v) for v in (0, 16, 32, 47) for u in (0, 24, 48, 72, 95)])
    wrong = {(48, 16), (72, 16), (48, 32), (72, 32)}  # a wrong prior around the right half
    D = np.array([shift + 9 if (int(u), int(v)) in wrong else shift for u, v in P], np.float32)
    tri = oracle_mod.delaunay(P)
    abc = oracle_mod.planes(P, D, tri)
    pidx = oracle_mod.raster(P, tri, W, H)
    Df = np.zeros((H, W), np.float32)
    Cf = np.full((H, W), 8, np.uint8)
    cells = oracle_mod.validate(cL, cR, om, pidx, abc, sz, Df, Cf, t_lo=4, t_hi=8)
    nb = int(cells["cb_w"].sum())
    assert nb >= 10  # the match branch is reached
    S_old = np.array([(u, v, d) for (u, v), d in zip(P.tolist(), D.tolist())], np.float64)
    S_new = oracle_mod.resample(cL, cR, sz, cells, S_old, dmax, t_lo=4, margin=2)
    old = {(int(u), int(v)): d for u, v, d in S_old}
    new = {(int(u), int(v)): d for u, v, d in S_new}
    # canonical order, no pixel twice, every old point kept as it was
    keys = [(int(v), int(u)) for u, v, _ in S_new]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    assert all(new[k] == d for k, d in old.items())
    cg_pix = {tuple(cells["cg_uv"][c]) for c in np.nonzero(cells["cg_w"])[0]}
    matched = 0
    for c in np.nonzero(cells["cb_w"])[0]:
        u, v = (int(x) for x in cells["cb_uv"][c])
        if (u, v) in old or (u, v) in cg_pix or u - shift < 2:
            continue
        # cost 0 at the true shift (closed form); the match takes it unless
        # another column in range also costs 0 before it, or one at distance
        # >= 2 costs less than 0 + margin (census codes of neighbouring pixels
        # are correlated, so this happens now and then)
        costs = [bin(int(cL[v, u]) ^ int(cR[v, u - d])).count("1") for d in range(min(dmax - 1, u - 2) + 1)]
        assert costs[shift] == 0
        unique = min(costs[:shift] + [99]) > 0 and all(c >= 2 for d, c in enumerate(costs) if abs(d - shift) >= 2)
        assert new.get((u, v)) == (shift if unique else None)
        matched += unique
    assert matched >= 10
    # nothing else joined: a C_g pick carries its D_it, a match the true shift
    cg_d = {tuple(int(x) for x in cells["cg_uv"][c]): float(cells["cg_d"][c]) for c in np.nonzero(cells["cg_w"])[0]}
    cb_pix = {tuple(int(x) for x in cells["cb_uv"][c]) for c in np.nonzero(cells["cb_w"])[0]}
    for k in set(new) - set(old):
        assert k in cg_d or k in cb_pix
        assert new[k] == (cg_d[k] if k in cg_d else shift)
