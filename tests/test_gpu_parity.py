"""Parity of the CUDA path (through the C ABI) with the CPU oracle, stage by
stage and end to end, on seeded synthetic pairs.  Integer outputs (census
codes, Omega_I bits, keypoints, matches, plane-index maps, costs, masks, cell
picks, support sets) must be bit-exact; interpolated fp32 disparities must
agree within 1e-3 px (the design target, and what is observed, is equality)."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on CPU machines, skipped there
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1511_00758_gb300 as S  # noqa: E402

DEV = "cuda:0"
TOL_D = 1e-3
PRM = dict(t_lo=4, t_hi=8, t_grad=8, t_fast=20, kp_per_bin=4, uniq_margin=2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    S.load()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _sync():
    torch.cuda.synchronize()


def _gpu_census(L, R, t_grad=8):
    H, W = L.shape
    cL = torch.empty((H, W), dtype=torch.int32, device=DEV)
    cR = torch.empty((H, W), dtype=torch.int32, device=DEV)
    om = torch.empty((H, (W + 31) // 32), dtype=torch.int32, device=DEV)
    S.census(_t(L), _t(R), W, H, t_grad, cL, cR, om)
    _sync()
    return cL, cR, om


def _unpack_omega(om, W):
    w = om.cpu().numpy().view(np.uint32)
    bits = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(w.shape[0], -1)
    return bits[:, :W].astype(np.uint8)


SIZES = [(77, 45), (640, 480), (1242, 375), (33, 9), (5, 5)]


@pytest.mark.parametrize("W,H", SIZES)
def test_census_omega(oracle_mod, W, H):
    rng = np.random.default_rng(W * 7 + H)
    L = rng.integers(0, 256, (H, W), dtype=np.uint8)
    R = np.clip(L.astype(int) + rng.integers(-20, 20, (H, W)), 0, 255).astype(np.uint8)
    cL, cR, om = _gpu_census(L, R)
    assert np.array_equal(cL.cpu().numpy().view(np.uint32), oracle_mod.census(L))
    assert np.array_equal(cR.cpu().numpy().view(np.uint32), oracle_mod.census(R))
    assert np.array_equal(_unpack_omega(om, W), oracle_mod.omega(L, 8))


def _gpu_fast(L, t_fast=20, K=4):
    H, W = L.shape
    scratch = torch.empty((H, W), dtype=torch.int16, device=DEV)
    out = torch.empty((120 * K, 2), dtype=torch.int32, device=DEV)
    S.fast(_t(L), W, H, t_fast, K, scratch, out)
    _sync()
    o = out.cpu().numpy()
    return o[o[:, 0] >= 0]


@pytest.mark.parametrize("name", ["vga_polygons", "driving_1242x375"])
def test_fast_bins_scene(oracle_mod, name):
    p = scenes.config_pairs(name)[0]
    assert np.array_equal(_gpu_fast(p.left), oracle_mod.fast_keypoints(p.left, 20, 4))


@pytest.mark.parametrize("K,t_fast,W,H", [(1, 10, 200, 90), (7, 15, 333, 101), (32, 5, 96, 70), (4, 20, 12, 10)])
def test_fast_bins_params(oracle_mod, K, t_fast, W, H):
    rng = np.random.default_rng(K + W)
    img = np.clip(scenes.value_noise(*np.meshgrid(np.arange(float(W)), np.arange(float(H))), 5 + K)
                  + rng.normal(0, 8, (H, W)), 0, 255).astype(np.uint8)
    assert np.array_equal(_gpu_fast(img, t_fast, K), oracle_mod.fast_keypoints(img, t_fast, K))


@pytest.mark.parametrize("dmax,t_lo,margin", [(64, 4, 2), (128, 12, 1), (256, 24, 3), (1, 4, 2), (37, 6, 0)])
def test_epipolar_match(oracle_mod, dmax, t_lo, margin):
    p = scenes.config_pairs("driving_1242x375")[0]
    H, W = p.left.shape
    cL, cR, _ = _gpu_census(p.left, p.right)
    rng = np.random.default_rng(dmax)
    q = np.stack([rng.integers(-3, W + 3, 3000), rng.integers(-3, H + 3, 3000)], 1).astype(np.int32)
    q[::50, 0] = -1
    out = torch.empty(len(q), dtype=torch.int32, device=DEV)
    S.epipolar_match(cL, cR, W, H, _t(q), len(q), dmax, t_lo, margin, out)
    _sync()
    want = oracle_mod.epipolar_match(oracle_mod.census(p.left), oracle_mod.census(p.right), q, dmax, t_lo, margin)
    assert np.array_equal(out.cpu().numpy(), want)


def _canon(P):
    P = np.asarray(P, np.int64)
    return np.ascontiguousarray(P[np.lexsort((P[:, 0], P[:, 1]))], dtype=np.int32)


def _tri_uv(P, tri):
    return np.ascontiguousarray(P[tri].reshape(-1, 6), dtype=np.int32)


def _gpu_raster(P, tri, W, H, abc=None):
    tuv = _tri_uv(P, tri)
    nbytes = S.raster_scratch_bytes(len(tri))
    scratch = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=DEV)
    pidx = torch.empty((H, W), dtype=torch.int32, device=DEV)
    dit = torch.empty((H, W), dtype=torch.float32, device=DEV) if abc is not None else None
    S.raster(_t(tuv) if len(tri) else None, _t(abc) if abc is not None and len(tri) else None, len(tri), W, H,
             pidx, dit, scratch, nbytes)
    _sync()
    return pidx.cpu().numpy(), (dit.cpu().numpy() if dit is not None else None)


def _same_f32(a, b):
    """Bit-identical fp32 maps (NaN where both are NaN)."""
    return np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[~np.isnan(a)].view(np.uint32),
                                                                        b[~np.isnan(b)].view(np.uint32))


@pytest.mark.parametrize("seed,n,W,H", [(1, 40, 640, 480), (2, 2000, 300, 200), (3, 6000, 257, 131),
                                        (4, 3, 50, 40), (5, 200, 1242, 375), (6, 30000, 1242, 375)])
def test_raster(oracle_mod, seed, n, W, H):
    rng = np.random.default_rng(seed)
    P = _canon(np.unique(np.stack([rng.integers(0, W, n), rng.integers(0, H, n)], 1), axis=0))
    D = rng.uniform(0, 100, len(P)).astype(np.float32)
    tri = oracle_mod.delaunay(P)
    abc = oracle_mod.planes(P, D, tri)
    want = oracle_mod.raster(P, tri, W, H)
    pidx, dit = _gpu_raster(P, tri, W, H, abc)
    assert np.array_equal(pidx, want)
    assert _same_f32(dit, oracle_mod.interp_map(want, abc))


def test_raster_empty_and_lattice(oracle_mod):
    W, H = 100, 60
    assert (_gpu_raster(np.zeros((0, 2), np.int32), np.zeros((0, 3), np.int32), W, H)[0] == -1).all()
    P = _canon([(u, v) for v in range(0, H, 3) for u in range(0, W, 4)])
    tri = oracle_mod.delaunay(P)
    got, _ = _gpu_raster(P, tri, W, H)
    assert np.array_equal(got, oracle_mod.raster(P, tri, W, H))


def _support_case(oracle_mod, p, n=400, seed=0):
    """A realistic mesh: the oracle's first support set plus random extra points on the ground truth."""
    H, W = p.left.shape
    r = oracle_mod.run(p.left, p.right, p.dmax, 1, 16, **PRM)
    S1 = r["support"][0]
    rng = np.random.default_rng(seed)
    extra = np.stack([rng.integers(0, W, n), rng.integers(0, H, n)], 1)
    pts = {(int(u), int(v)): float(d) for u, v, d in S1}
    for u, v in extra:
        pts.setdefault((int(u), int(v)), float(np.float32(p.gt_disp[v, u] + rng.normal(0, 0.7))))
    keys = sorted(pts, key=lambda t: (t[1], t[0]))
    P = np.array(keys, np.int32)
    D = np.array([pts[k] for k in keys], np.float32)
    return P, D


@pytest.mark.parametrize("bulk", [0, 1])
@pytest.mark.parametrize("name,sz,first", [("vga_polygons", 16, 1), ("driving_1242x375", 8, 0),
                                           ("driving_1242x375", 1, 0), ("vga_polygons", 3, 0),
                                           ("driving_1242x375", 64, 1), ("driving_1242x375", 4, 0),
                                           ("vga_polygons", 2, 1), ("driving_1242x375", 6, 0),
                                           ("vga_polygons", 12, 0), ("driving_1242x375", 5, 0),
                                           ("vga_polygons", 40, 0), ("driving_1242x375", 7, 1)])
def test_validate(oracle_mod, name, sz, first, bulk):
    p = scenes.config_pairs(name)[0]
    H, W = p.left.shape
    P, D = _support_case(oracle_mod, p)
    tri = oracle_mod.delaunay(P)
    abc = oracle_mod.planes(P, D, tri)
    pidx = oracle_mod.raster(P, tri, W, H)
    cL_o, cR_o, om_o = oracle_mod.census(p.left), oracle_mod.census(p.right), oracle_mod.omega(p.left)
    rng = np.random.default_rng(sz)
    Df0 = rng.uniform(0, 50, (H, W)).astype(np.float32)
    Cf0 = rng.integers(0, 12, (H, W)).astype(np.uint8)
    if first:
        Df0[:] = 0
        Cf0[:] = PRM["t_hi"]
    Df_o, Cf_o = Df0.copy(), Cf0.copy()
    ro = oracle_mod.validate(cL_o, cR_o, om_o, pidx, abc, sz, Df_o, Cf_o, PRM["t_lo"], PRM["t_hi"])

    cL, cR, om = _gpu_census(p.left, p.right)
    dit = _t(oracle_mod.interp_map(pidx, abc))
    Df = _t(Df0 if not first else np.full((H, W), 7.0, np.float32))
    Cf = _t(Cf0 if not first else np.full((H, W), 3, np.uint8))
    mask = torch.empty((H, W), dtype=torch.uint8, device=DEV)
    nc = ro["Wc"] * ro["Hc"]
    cg = torch.full((nc,), -1, dtype=torch.int32, device=DEV)
    cb = torch.full((nc,), -1, dtype=torch.int32, device=DEV)
    if bulk:
        err = torch.zeros(1, dtype=torch.int32, device=DEV)
        S.validate_bulk(cL, cR, om, dit, W, H, sz, PRM["t_lo"], PRM["t_hi"], first, Df, Cf, mask, cg, cb, err)
        _sync()
        assert int(err.item()) == 0
    else:
        S.validate(cL, cR, om, dit, W, H, sz, PRM["t_lo"], PRM["t_hi"], first, Df, Cf, mask, cg, cb)
    _sync()
    assert np.array_equal(mask.cpu().numpy(), ro["mask"])
    assert np.array_equal(Cf.cpu().numpy(), Cf_o)
    dd = Df.cpu().numpy()
    assert np.abs(dd - Df_o).max() <= TOL_D
    assert np.array_equal(dd.view(np.uint32), Df_o.view(np.uint32))
    g = cg.cpu().numpy().view(np.uint32)
    b = cb.cpu().numpy().view(np.uint32)
    IDX = (1 << 27) - 1
    assert np.array_equal(g != 0xFFFFFFFF, ro["cg_w"] == 1)
    assert np.array_equal(b != 0xFFFFFFFF, ro["cb_w"] == 1)
    wg = ro["cg_w"] == 1
    assert np.array_equal((g[wg] & IDX) % W, ro["cg_uv"][wg, 0]) and np.array_equal((g[wg] & IDX) // W, ro["cg_uv"][wg, 1])
    assert np.array_equal(g[wg] >> 27, ro["cg_cost"][wg])
    wb = ro["cb_w"] == 1
    assert np.array_equal((b[wb] & IDX) % W, ro["cb_uv"][wb, 0]) and np.array_equal((b[wb] & IDX) // W, ro["cb_uv"][wb, 1])
    assert np.array_equal(24 - (b[wb] >> 27), ro["cb_cost"][wb])
    assert wg.sum() > 10 and (wb.sum() > 10 or sz > 8)

    # resample + match on the same cells
    cgd = torch.empty(nc, dtype=torch.float32, device=DEV)
    xd = torch.empty(nc, dtype=torch.int32, device=DEV)
    dmax = p.dmax
    S.resample_match(cg, cb, nc, dit, cL, cR, W, H, dmax, PRM["t_lo"], PRM["uniq_margin"], cgd, xd)
    _sync()
    cgd = cgd.cpu().numpy()
    assert np.isnan(cgd[~wg]).all()
    assert np.array_equal(cgd[wg].view(np.uint32), ro["cg_d"][wg].view(np.uint32))
    want = np.full(nc, -1, np.int32)
    if wb.any():
        want[wb] = oracle_mod.epipolar_match(cL_o, cR_o, ro["cb_uv"][wb], dmax, PRM["t_lo"], PRM["uniq_margin"])
    assert np.array_equal(xd.cpu().numpy(), want)


def _run_ctx(pairs, max_slots=1, host_threads=1, budget=1 << 30, window_us=0, prm=PRM, host_mesh=0):
    with S.Context(mem_budget_bytes=budget, max_slots=max_slots, host_threads=host_threads,
                   batch_window_us=window_us, host_mesh=host_mesh, **prm) as ctx:
        tickets = [ctx.submit(_t(p.left), _t(p.right), p.left.shape[1], p.left.shape[0], p.dmax, p.iters, p.cell)
                   for p in pairs]
        outs = []
        for t in tickets:
            r = ctx.poll(t)
            outs.append(ctx.result_tensors(r))
            ctx.release(t)
        return outs


def _compare_run(oracle_mod, p, got, prm=PRM):
    want = oracle_mod.run(p.left, p.right, p.dmax, p.iters, p.cell, **prm)
    assert [len(s) for s in got["support"]] == [len(s) for s in want["support"]]
    for a, b in zip(got["support"], want["support"]):
        assert np.array_equal(a[:, :2], b[:, :2])
        assert np.array_equal(a[:, 2].astype(np.float32).view(np.uint32), b[:, 2].astype(np.float32).view(np.uint32))
    assert list(got["n_tri"]) == list(want["n_tri"])
    assert np.array_equal(got["planeidx"].cpu().numpy(), want["planeidx"])
    assert np.array_equal(got["mask"].cpu().numpy(), want["mask"])
    assert np.array_equal(got["C_f"].cpu().numpy(), want["C_f"])
    dd = got["D_f"].cpu().numpy()
    assert np.abs(dd - want["D_f"]).max() <= TOL_D
    return want


@pytest.mark.parametrize("name", ["vga_polygons", "driving_1242x375"])
def test_end_to_end_dense(oracle_mod, name):
    """The dense variant (t_grad = 0: every pixel inside the 2-pixel border is
    evaluated) through the engine, against the oracle run with the same setting."""
    prm = dict(PRM, t_grad=0)
    p = scenes.config_pairs(name)[0]
    want = _compare_run(oracle_mod, p, _run_ctx([p], prm=prm)[0], prm=prm)
    H, W = p.left.shape
    assert (want["mask"][2:H - 2, 2:W - 2] & 1).all()  # all of the interior is in Omega


def test_end_to_end_autotuned(oracle_mod):
    """A context that tunes its kernels' work shapes at create gives the same
    results (the shapes only move time)."""
    p = scenes.config_pairs("driving_1242x375")[0]
    H, W = p.left.shape
    with S.Context(mem_budget_bytes=1 << 30, max_slots=1, host_threads=1, autotune=1, tune_w=W, tune_h=H,
                   **PRM) as ctx:
        tu = ctx.tuning()
        assert tu["autotuned"] == 1 and tu["raster_us"] > 0 and tu["validate_us"] > 0
        assert tu["small_area"] in (128, 256, 512) and tu["batch_area"] in (512, 1024, 2048)
        assert tu["raster_cols"] in (64, 128, 256) and tu["validate_blocks_per_sm"] in (4, 8, 16)
        t = ctx.submit(_t(p.left), _t(p.right), W, H, p.dmax, p.iters, p.cell)
        got = ctx.result_tensors(ctx.poll(t))
        ctx.release(t)
    _compare_run(oracle_mod, p, got)


def test_end_to_end_idle_workers_and_round_shapes(oracle_mod):
    """Four host workers on one driving pair: the idle ones take halves of the
    large triangulations (same triangles, so the same results), and each round
    launches only the stage it has work for (the raster also resets the cell
    records, so neither the clear nor the reset has launches of its own)."""
    p = scenes.config_pairs("driving_1242x375")[0]
    H, W = p.left.shape
    with S.Context(mem_budget_bytes=1 << 30, max_slots=1, host_threads=4, host_mesh=1, **PRM) as ctx:
        t = ctx.submit(_t(p.left), _t(p.right), W, H, p.dmax, p.iters, p.cell)
        got = ctx.result_tensors(ctx.poll(t))
        ctx.release(t)
        st = ctx.stats()
    want = _compare_run(oracle_mod, p, got)
    assert max(len(s) for s in want["support"]) >= 4096  # large enough to fork
    k = list(st.kind_launches)
    assert k[0:4] == [1, 1, 1, 1]  # one seed round
    assert k[5] == k[6] == k[7] == p.iters  # one iteration round per pass
    assert k[4] == 0 and k[8] == 0 and k[9] == 0
    assert st.gpu_rounds == 1 + p.iters


@pytest.mark.parametrize("host_mesh", [0, 1])
def test_end_to_end_mesh_paths(oracle_mod, host_mesh):
    """Both mesh paths on one driving pair: the host triangulating every pass,
    or only the first pass's mesh on the host and each later one re-tessellated
    on the device (one mesh launch per resampling pass, no host step between
    passes).  Both equal the oracle."""
    p = scenes.config_pairs("driving_1242x375")[0]
    H, W = p.left.shape
    with S.Context(mem_budget_bytes=1 << 30, max_slots=1, host_threads=2, host_mesh=host_mesh, **PRM) as ctx:
        t = ctx.submit(_t(p.left), _t(p.right), W, H, p.dmax, p.iters, p.cell)
        got = ctx.result_tensors(ctx.poll(t))
        ctx.release(t)
        st = ctx.stats()
    _compare_run(oracle_mod, p, got)
    k = list(st.kind_launches)
    assert k[5] == k[6] == k[7] == p.iters
    assert k[9] == (0 if host_mesh else p.iters - 1)
    assert st.gpu_rounds == 1 + p.iters


def test_end_to_end_vga_one_iteration(oracle_mod):
    p = scenes.config_pairs("vga_polygons")[0]
    want = _compare_run(oracle_mod, p, _run_ctx([p])[0])
    assert (want["C_f"] < 8).mean() > 0.2


def test_end_to_end_driving_full_size(oracle_mod):
    """The 1242x375 driving workload at full size, 3 iterations, 8x8 cells."""
    p = scenes.config_pairs("driving_1242x375")[0]
    want = _compare_run(oracle_mod, p, _run_ctx([p])[0])
    assert len(want["support"][2]) > len(want["support"][1]) > len(want["support"][0])


@pytest.mark.parametrize("W,H,dmax,iters,cell", [(321, 123, 48, 4, 16), (97, 61, 16, 3, 1), (200, 100, 1, 2, 4)])
def test_end_to_end_ragged(oracle_mod, W, H, dmax, iters, cell):
    pr = scenes.make_pair("polygon", W, H, 99 + W, min(dmax, 64), iters, cell, n_poly=6, sigma=2.0)
    pr.dmax = dmax
    _compare_run(oracle_mod, pr, _run_ctx([pr])[0])


def test_end_to_end_degenerate(oracle_mod):
    # flat images: no corners, no Omega_I, no mesh; D_f = 0 and C_f = t_hi everywhere
    flat = scenes.StereoPair(np.full((40, 70), 100, np.uint8), np.full((40, 70), 100, np.uint8),
                             np.zeros((40, 70), np.float32), np.zeros((40, 70), bool), 32, 3, 8)
    got = _run_ctx([flat])[0]
    _compare_run(oracle_mod, flat, got)
    assert (got["C_f"].cpu().numpy() == 8).all() and (got["D_f"].cpu().numpy() == 0).all()
    tiny = scenes.StereoPair(np.random.default_rng(1).integers(0, 256, (5, 5), dtype=np.uint8),
                             np.random.default_rng(2).integers(0, 256, (5, 5), dtype=np.uint8),
                             np.zeros((5, 5), np.float32), np.zeros((5, 5), bool), 4, 2, 1)
    _compare_run(oracle_mod, tiny, _run_ctx([tiny])[0])


def test_end_to_end_bulk_validate(oracle_mod, monkeypatch):
    """The engine with the bulk-copy validate kernel gives the same results."""
    monkeypatch.setenv("STEREO_VALIDATE", "bulk")
    p = scenes.config_pairs("driving_1242x375")[0]
    _compare_run(oracle_mod, p, _run_ctx([p])[0])


def test_batched_serving_matches_solo(oracle_mod):
    """Continuous batching: results in a mixed batch equal solo results bit for bit."""
    pairs = [scenes.make_pair("polygon", 320, 240, 500 + i, 64, 3, 16, n_poly=10) for i in range(3)]
    pairs += [scenes.make_pair("driving", 400, 150, 600 + i, 96, 2, 8, n_box=10) for i in range(3)]
    solo = [_run_ctx([p], host_mesh=1)[0] for p in pairs]  # host meshes, one pair at a time
    for slots, threads, window in ((4, 3, 0), (6, 2, 2000)):
        mixed = _run_ctx(pairs, max_slots=slots, host_threads=threads, window_us=window)  # device meshes, batched
        for a, b in zip(solo, mixed):
            for k in ("D_f", "C_f", "mask", "planeidx"):
                assert torch.equal(a[k], b[k]), k
            for x, y in zip(a["support"], b["support"]):
                assert np.array_equal(x, y)


def test_batched_mixed_cell_classes(oracle_mod):
    """One batch whose pairs fall in every fused-validate class over their passes
    (cell sides 5, 12, 2 and 3 halve to 6, 2, 1, 1 ...): batched equals solo bit
    for bit, and one pair equals the oracle."""
    pairs = [scenes.make_pair("polygon", 200, 120, 700 + i, 48, 3, cell, n_poly=8)
             for i, cell in enumerate((5, 12, 2, 3))]
    solo = [_run_ctx([p])[0] for p in pairs]
    mixed = _run_ctx(pairs, max_slots=4, host_threads=2)
    for a, b in zip(solo, mixed):
        for k in ("D_f", "C_f", "mask", "planeidx"):
            assert torch.equal(a[k], b[k]), k
    _compare_run(oracle_mod, pairs[1], mixed[1])


def test_host_input_pointers(oracle_mod):
    """Host inputs, and the result delivered to host buffers by poll_host (pageable
    numpy arrays and page-locked tensors) equal to the device result."""
    p = scenes.config_pairs("vga_polygons")[0]
    with S.Context(mem_budget_bytes=1 << 28, **PRM) as ctx:
        t = ctx.submit(p.left, p.right, 640, 480, p.dmax, p.iters, p.cell)
        got = ctx.result_tensors(ctx.poll(t))
        d = np.full((480, 640), -7.0, np.float32)
        c = np.zeros((480, 640), np.uint8)
        m = np.zeros((480, 640), np.uint8)
        r = ctx.poll_host(t, d, c, m)
        assert r.status == 0 and r.w == 640
        dp = torch.empty((480, 640), dtype=torch.float32).pin_memory()
        cp = torch.empty((480, 640), dtype=torch.uint8).pin_memory()
        ctx.poll_host(t, dp, cp)  # the mask skipped
        ctx.release(t)
    assert np.array_equal(d.view(np.uint32), got["D_f"].cpu().numpy().view(np.uint32))
    assert np.array_equal(c, got["C_f"].cpu().numpy()) and np.array_equal(m, got["mask"].cpu().numpy())
    assert np.array_equal(dp.numpy().view(np.uint32), d.view(np.uint32)) and np.array_equal(cp.numpy(), c)
    _compare_run(oracle_mod, p, got)


def test_pinned_host_input_pointers(oracle_mod):
    """Page-locked host inputs take the direct-copy path; the caller may reuse
    them as soon as submit returns."""
    p = scenes.config_pairs("vga_polygons")[0]
    left = torch.from_numpy(p.left.copy()).pin_memory()
    right = torch.from_numpy(p.right.copy()).pin_memory()
    with S.Context(mem_budget_bytes=1 << 28, **PRM) as ctx:
        t = ctx.submit(left, right, 640, 480, p.dmax, p.iters, p.cell)
        left.zero_()
        right.zero_()  # overwritten right after submit: the request already holds its copy
        got = ctx.result_tensors(ctx.poll(t))
        ctx.release(t)
    _compare_run(oracle_mod, p, got)


def test_result_destinations_at_submit(oracle_mod):
    """Results written to the caller's buffers named at submit, in the round that
    finishes each request: page-locked host tensors, pageable numpy arrays, device
    tensors and a partial set (D_f only), in one batch with device-mesh and
    mixed sizes; each equals the request's own device result.  Page-locked inputs
    are read by the copy kernel and may be reused at once."""
    pairs = scenes.config_pairs("vga_polygons", n=2) + [scenes.make_pair("driving", 400, 150, 611, 96, 3, 8, n_box=10)]
    outs = []
    for i, p in enumerate(pairs):
        H, W = p.left.shape
        if i == 0:
            o = (torch.full((H, W), -7.0).pin_memory(), torch.zeros((H, W), dtype=torch.uint8).pin_memory(),
                 torch.zeros((H, W), dtype=torch.uint8).pin_memory())
        elif i == 1:
            o = (np.full((H, W), -7.0, np.float32), np.zeros((H, W), np.uint8), np.zeros((H, W), np.uint8))
        else:
            o = (torch.full((H, W), -7.0, device=DEV), None, None)
        outs.append(o)
    ins = [(torch.from_numpy(p.left.copy()).pin_memory(), torch.from_numpy(p.right.copy()).pin_memory()) for p in pairs]
    with S.Context(mem_budget_bytes=1 << 30, max_slots=3, host_threads=2, **PRM) as ctx:
        tk = ctx.submit_batch([(l, r, p.left.shape[1], p.left.shape[0], p.dmax, p.iters, p.cell, 0, o)
                               for (l, r), p, o in zip(ins, pairs, outs)])
        assert len(tk) == 3
        for l, r in ins:
            l.zero_()
            r.zero_()
        got = []
        for t in tk:
            got.append(ctx.result_tensors(ctx.poll(t)))
            ctx.release(t)
    torch.cuda.synchronize()

    def host(x):
        return x.cpu().numpy() if torch.is_tensor(x) else x

    for o, g in zip(outs, got):
        assert np.array_equal(host(o[0]).view(np.uint32), g["D_f"].cpu().numpy().view(np.uint32))
        if o[1] is not None:
            assert np.array_equal(host(o[1]), g["C_f"].cpu().numpy())
            assert np.array_equal(host(o[2]), g["mask"].cpu().numpy())
    _compare_run(oracle_mod, pairs[0], got[0])


def test_budget_errors():
    with S.Context(mem_budget_bytes=1 << 22, **PRM) as ctx:
        img = np.zeros((480, 640), np.uint8)
        with pytest.raises(S.StereoError) as e:
            ctx.submit(img, img, 640, 480, 64, 1, 16)
        assert e.value.code == -2
        with pytest.raises(S.StereoError) as e:
            ctx.submit(img, img, 640, 480, 300, 1, 16)
        assert e.value.code == -1
