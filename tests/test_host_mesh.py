"""CPU-side checks of libstereo: it loads and exports every entry point the
header declares; the host mesh step (Guibas-Stolfi Delaunay + plane solve)
agrees exactly with the oracle's independent gift-wrapping triangulation and
plane solve; argument errors are reported before anything is launched."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1511_00758_gb300 as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    return S.load()


def test_exports_every_declared_symbol(L):
    hdr = open(os.path.join(ROOT, "include", "stereo.h")).read()
    names = set(re.findall(r"^\s*(?:[\w\*]+\s+)+\**(stereo_\w+)\s*\(", hdr, re.M))
    assert len(names) >= 16
    for n in names:
        assert hasattr(L, n), n
    assert set(S.SYMBOLS) <= names


def _canon(P):
    P = np.asarray(P, np.int64)
    return np.ascontiguousarray(P[np.lexsort((P[:, 0], P[:, 1]))], dtype=np.int32)


def _lib_delaunay(P):
    n = len(P)
    cap = 2 * n + 8
    tri = np.zeros((cap, 3), np.int32)
    T = S.delaunay(P, n, tri, cap)
    return tri[:T]


@pytest.mark.parametrize("seed,n,span", [(1, 50, 1000), (2, 400, 16000), (3, 300, 30), (4, 200, 12),
                                         (5, 1500, 200), (6, 64, 8)])
def test_delaunay_matches_oracle(oracle_mod, seed, n, span):
    rng = np.random.default_rng(seed)
    P = _canon(np.unique(rng.integers(0, span, (n, 2)), axis=0))
    assert np.array_equal(_lib_delaunay(P), oracle_mod.delaunay(P))


def test_delaunay_full_lattice_and_lines(oracle_mod):
    P = _canon([(u, v) for v in range(0, 40, 2) for u in range(0, 60, 3)])
    assert np.array_equal(_lib_delaunay(P), oracle_mod.delaunay(P))
    line = _canon([(u, 7) for u in range(20)])
    assert len(_lib_delaunay(line)) == 0 and len(oracle_mod.delaunay(line)) == 0
    P = _canon([(u, 3) for u in range(10)] + [(4, 9)])
    assert np.array_equal(_lib_delaunay(P), oracle_mod.delaunay(P))


def test_delaunay_support_like_points(oracle_mod):
    """Cell-sampled points as resampling produces them: one or two per cell, many cocircular."""
    rng = np.random.default_rng(9)
    pts = set()
    for cy in range(0, 120, 8):
        for cx in range(0, 200, 8):
            for _ in range(rng.integers(0, 3)):
                pts.add((cx + int(rng.integers(0, 8)), cy + int(rng.integers(0, 8))))
    P = _canon(sorted(pts))
    assert np.array_equal(_lib_delaunay(P), oracle_mod.delaunay(P))


def _lattice_points(seed, w, h, step):
    rng = np.random.default_rng(seed)
    pts = {(min(w - 1, u + int(rng.integers(0, step))), min(h - 1, v + int(rng.integers(0, step))))
           for v in range(0, h, step) for u in range(0, w, step)}
    return _canon(sorted(pts))


@pytest.mark.parametrize("threads", [2, 4, 8])
def test_delaunay_parallel_matches_serial(oracle_mod, threads):
    """The forked top splits (halves of 2048 points or more) give the serial triangulation."""
    P = _lattice_points(30 + threads, 1242, 375, 7)  # about 9500 points: three forked levels
    n = len(P)
    cap = 2 * n + 8
    tri = np.zeros((cap, 3), np.int32)
    T = S.delaunay_parallel(P, n, tri, cap, threads)
    serial = _lib_delaunay(P)
    assert T == len(serial) and np.array_equal(tri[:T], serial)
    if threads == 8:  # and the oracle's gift wrapping, once
        assert np.array_equal(serial, oracle_mod.delaunay(P))


def test_delaunay_parallel_degenerate_sets():
    """Forked splits on degenerate sets give the serial triangulation: a full
    lattice (every square cocircular), three long collinear rows, and all
    points on one line (no triangle)."""
    lattice = _canon([(u, v) for v in range(0, 300, 3) for u in range(0, 420, 3)])  # 14000 points
    rows = _canon([(u, v) for v in (0, 1, 57) for u in range(0, 3000)])
    line = _canon([(u, 5) for u in range(9000)])
    for P in (lattice, rows, line):
        n = len(P)
        cap = 2 * n + 8
        serial = _lib_delaunay(P)
        for threads in (2, 8):
            tri = np.zeros((cap, 3), np.int32)
            T = S.delaunay_parallel(P, n, tri, cap, threads)
            assert T == len(serial) and np.array_equal(tri[:T], serial)
    assert len(_lib_delaunay(line)) == 0


def test_planes_bit_exact(oracle_mod):
    rng = np.random.default_rng(10)
    P = _canon(np.unique(rng.integers(0, 300, (200, 2)), axis=0))
    D = rng.uniform(0, 100, len(P)).astype(np.float32)
    D[::3] = np.rint(D[::3])
    tri = oracle_mod.delaunay(P)
    abc = np.zeros((len(tri), 3), np.float32)
    S.planes(P, D, np.ascontiguousarray(tri), len(tri), abc)
    assert np.array_equal(abc.view(np.uint32), oracle_mod.planes(P, D, tri).view(np.uint32))


def test_host_argument_errors(L):
    P = np.array([[5, 5], [1, 5], [3, 9]], np.int32)  # not canonical: (1,5) must come first
    tri = np.zeros((8, 3), np.int32)
    assert L.stereo_delaunay(P.ctypes.data, 3, tri.ctypes.data, 8) == -1
    assert L.stereo_delaunay_parallel(P.ctypes.data, 3, tri.ctypes.data, 8, 4) == -1
    Q = np.ascontiguousarray(P[[1, 0, 2]])
    assert L.stereo_delaunay_parallel(Q.ctypes.data, 3, tri.ctypes.data, 8, 0) == -1  # threads < 1
    assert L.stereo_delaunay_parallel(Q.ctypes.data, 3, tri.ctypes.data, 8, 2) == 1
    assert L.stereo_census(None, None, 64, 64, 8, None, None, None, None) == -1
    assert L.stereo_census(1, 1, 3, 64, 8, None, None, None, None) == -1
    assert L.stereo_epipolar_match(1, 1, 64, 64, 1, 4, 300, 4, 2, 1, None) == -1
    assert L.stereo_validate(1, 1, 1, 1, 1, 64, 64, 4, 9, 8, 1, 1, 1, None, 1, None, None) == -1
    assert L.stereo_validate(1, 1, 1, 1, 64, 64, 8, 4, 8, 0, 1, 1, None, None, None, None) == -1  # mask required
    assert L.stereo_submit(None, 0, None, None, 64, 64, 64, 1, 16, ctypes.byref(ctypes.c_uint64())) == -1
    cfg = S.Config()
    L.stereo_default_config(ctypes.byref(cfg))
    assert (cfg.t_lo, cfg.t_hi, cfg.kp_per_bin, cfg.uniq_margin) == (4, 8, 4, 2)
    cfg.t_lo = 20
    h = ctypes.c_void_p()
    assert L.stereo_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
