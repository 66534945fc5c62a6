"""End-to-end parity at the large frame sizes: 1280x720 and 1920x1080 (dmax 128,
2 iterations, 16x16 cells) and 2048x1536 with dmax 256 (3 iterations) against
the oracle; and the full large workload (2048x1536, dmax 256, 5 iterations,
4x4 cells down to 1x1, millions of support points, beyond the oracle's
quadratic triangulation) checked on sampled pixels against values the oracle
computes one by one, and for equality between the device-mesh and host-mesh
paths; and the driving workload's whole 64-pair batch in one submission, device
meshes against host meshes."""
from fractions import Fraction

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1511_00758_gb300 as S  # noqa: E402

PRM = dict(t_lo=4, t_hi=8, t_grad=8, t_fast=20, kp_per_bin=4, uniq_margin=2)
TOL_D = 1e-3
SEED = 0x5EED0000 + 7000


def _f32(x):
    """An exact rational rounded to the nearest float32 (ties to even)."""
    x = Fraction(x)
    if x == 0:
        return Fraction(0)
    sign, a = (-1 if x < 0 else 1), abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while a >= Fraction(2) ** (e + 1):
        e += 1
    while a < Fraction(2) ** e:
        e -= 1
    q = a / Fraction(2) ** (e - 23)
    n = q.numerator // q.denominator
    r = q - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return sign * Fraction(n) * Fraction(2) ** (e - 23)


def _fma_plane(abc, u, v):
    """fma(a, u, fma(b, v, c)) in fp32: each fma rounded once."""
    a, b, c = (Fraction(float(x)) for x in abc)
    return float(_f32(a * u + _f32(b * v + c)))


def _run(p, host_mesh=0, budget=8 << 30):
    H, W = p.left.shape
    with S.Context(mem_budget_bytes=budget, max_slots=1, host_threads=4, host_mesh=host_mesh, **PRM) as ctx:
        t = ctx.submit(torch.from_numpy(p.left).cuda(), torch.from_numpy(p.right).cuda(), W, H, p.dmax, p.iters,
                       p.cell)
        out = ctx.result_tensors(ctx.poll(t))
        ctx.release(t)
    return out


def _compare(oracle_mod, p, got):
    want = oracle_mod.run(p.left, p.right, p.dmax, p.iters, p.cell, **PRM)
    assert [len(s) for s in got["support"]] == [len(s) for s in want["support"]]
    for a, b in zip(got["support"], want["support"]):
        assert np.array_equal(a[:, :2], b[:, :2])
        assert np.array_equal(a[:, 2].astype(np.float32).view(np.uint32), b[:, 2].astype(np.float32).view(np.uint32))
    assert list(got["n_tri"]) == list(want["n_tri"])
    assert np.array_equal(got["planeidx"].cpu().numpy(), want["planeidx"])
    assert np.array_equal(got["mask"].cpu().numpy(), want["mask"])
    assert np.array_equal(got["C_f"].cpu().numpy(), want["C_f"])
    assert np.abs(got["D_f"].cpu().numpy() - want["D_f"]).max() <= TOL_D


@pytest.mark.parametrize("W,H,seed", [(1280, 720, 1), (1920, 1080, 2)])
def test_end_to_end_hd_sizes(oracle_mod, W, H, seed):
    p = scenes.make_pair("polygon", W, H, SEED + seed, 128, 2, 16, n_poly=20, sigma=2.0)
    _compare(oracle_mod, p, _run(p))


def test_end_to_end_2048x1536_dmax256(oracle_mod):
    p = scenes.make_pair("polygon", 2048, 1536, SEED + 3, 256, 3, 16, n_poly=30, sigma=2.0)
    got = _run(p)
    _compare(oracle_mod, p, got)
    assert (got["C_f"].cpu().numpy() < 8).mean() > 0.1


def test_full_large_workload_sampled(oracle_mod):
    """2048x1536, dmax 256, 5 iterations from 4x4 cells: the device-mesh path
    equals the host-mesh path (an independent triangulation, itself equal to
    the oracle's), and sampled pixels satisfy what the oracle fixes one by one:
    the last pass's plane-index map names the triangle of the canonical
    triangulation of S_5 that the fill rule gives the pixel, D_it is that
    triangle's plane at the pixel, and every validated pixel's C_f is the
    census cost of its stored disparity."""
    p = scenes.large_pairs(n=1)[0]
    H, W = p.left.shape
    got = _run(p)
    ref = _run(p, host_mesh=1)
    for k in ("D_f", "C_f", "mask", "planeidx"):
        assert torch.equal(got[k], ref[k]), k
    assert list(got["n_tri"]) == list(ref["n_tri"])
    for a, b in zip(got["support"], ref["support"]):
        assert np.array_equal(a, b)
    S5 = got["support"][-1]
    assert len(S5) > 500000
    P = np.ascontiguousarray(S5[:, :2].astype(np.int32))
    tri = np.zeros((2 * len(P) + 8, 3), np.int32)
    T = S.delaunay(P, len(P), tri, len(tri))
    assert T == int(got["n_tri"][-1])
    tri = tri[:T]
    pidx = got["planeidx"].cpu().numpy()
    mask = got["mask"].cpu().numpy()
    Df = got["D_f"].cpu().numpy()
    Cf = got["C_f"].cpu().numpy()
    rng = np.random.default_rng(77)
    us, vs = rng.integers(0, W, 3000), rng.integers(0, H, 3000)
    cover = [(u, v) for u, v in zip(us, vs) if pidx[v, u] >= 0][:400]
    assert len(cover) > 300
    for u, v in cover:  # the pixel lies in its triangle (fill rule) and D_it is the plane there
        t = int(pidx[v, u])
        Pt = np.ascontiguousarray(P[tri[t]])
        one = np.array([[0, 1, 2]], np.int32)
        assert oracle_mod.raster(Pt, one, W, H)[v, u] == 0
        abc = oracle_mod.planes(Pt, S5[tri[t], 2].astype(np.float32), one)[0]
        k = int(np.rint(_fma_plane(abc, u, v)))
        if mask[v, u] & 1:
            assert bool(mask[v, u] & 2) == (2 <= u - k <= W - 3)
    cL, cR = oracle_mod.census(p.left), oracle_mod.census(p.right)
    val = np.argwhere(Cf < 8)
    pick = val[rng.choice(len(val), 2000, replace=False)]
    for v, u in pick:
        k = int(np.rint(Df[v, u]))
        assert bin(int(cL[v, u]) ^ int(cR[v, u - k])).count("1") == Cf[v, u]


def _run_batch(pairs, host_mesh):
    H, W = pairs[0].left.shape
    p0 = pairs[0]
    need = len(pairs) * S.request_bytes(W, H, p0.dmax, p0.iters, p0.cell)
    with S.Context(mem_budget_bytes=(1 << 29) + need, max_slots=len(pairs), max_queue=2 * len(pairs),
                   host_threads=8, host_mesh=host_mesh, **PRM) as ctx:
        ins = [(torch.from_numpy(p.left).cuda(), torch.from_numpy(p.right).cuda()) for p in pairs]
        outs = []
        for rep in range(1 if host_mesh else 3):
            tickets = ctx.submit_batch([(l, r, W, H, p.dmax, p.iters, p.cell) for (l, r), p in zip(ins, pairs)])
            assert len(tickets) == len(pairs)
            run = []
            for t in tickets:
                res = ctx.poll(t)
                assert res.status == 0
                run.append(ctx.result_tensors(res))
                ctx.release(t)
            outs.append(run)
        return outs


def test_full_batch_device_mesh_equals_host_mesh():
    """64 pairs of 1242x375 (the driving workload's whole batch) in one submission:
    each device mesh pass runs 64 thread-block clusters of several blocks, whose
    insertion and flip rounds share worklists and counters across the blocks of a
    cluster.  Three repetitions of the batch equal the host-mesh path bit for bit."""
    pairs = scenes.config_pairs("driving_1242x375", n=64)
    ref = _run_batch(pairs, host_mesh=1)[0]
    for run in _run_batch(pairs, host_mesh=0):
        for a, b in zip(ref, run):
            for k in ("D_f", "C_f", "mask", "planeidx"):
                assert torch.equal(a[k], b[k]), k
            assert list(a["n_tri"]) == list(b["n_tri"])
            for x, y in zip(a["support"], b["support"]):
                assert np.array_equal(x, y)
