"""CPU oracle of the iterative stereo method (Alg. 1-4), as a ctypes wrapper.

TEST INFRASTRUCTURE ONLY: the parity tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  The product library never imports,
links or calls anything here.  The arithmetic lives in ``oracle.c`` (plain C,
single thread, ``-ffp-contract=off``); this module only compiles it and
marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_lib")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None

DEFAULT_PARAMS = dict(t_lo=4, t_hi=8, t_grad=8, t_fast=20, kp_per_bin=4, uniq_margin=2)


class _Params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("t_lo", "t_hi", "t_grad", "t_fast", "kp_per_bin", "uniq_margin")]


def build(force=False):
    """Compile oracle.c into a shared library (gcc, portable flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def census(img):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    out = np.zeros((H, W), np.uint32)
    lib().or_census(_p(img), W, H, _p(out))
    return out


def omega(L, t_grad=DEFAULT_PARAMS["t_grad"]):
    L = np.ascontiguousarray(L, dtype=np.uint8)
    H, W = L.shape
    out = np.zeros((H, W), np.uint8)
    lib().or_omega(_p(L), W, H, int(t_grad), _p(out))
    return out


def fast_score(img, u, v, t_fast=DEFAULT_PARAMS["t_fast"]):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    return lib().or_fast_score(_p(img), W, H, int(u), int(v), int(t_fast))


def fast_keypoints(img, t_fast=DEFAULT_PARAMS["t_fast"], K=DEFAULT_PARAMS["kp_per_bin"]):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    cap = 120 * max(K, 1)
    out = np.zeros((cap, 2), np.int32)
    n = lib().or_fast_keypoints(_p(img), W, H, int(t_fast), int(K), _p(out), cap)
    if n < 0:
        raise RuntimeError(f"or_fast_keypoints failed: {n}")
    return out[:n].copy()


def epipolar_match(cL, cR, q_uv, dmax, t_lo=DEFAULT_PARAMS["t_lo"], margin=DEFAULT_PARAMS["uniq_margin"]):
    cL = np.ascontiguousarray(cL, dtype=np.uint32)
    cR = np.ascontiguousarray(cR, dtype=np.uint32)
    q = np.ascontiguousarray(q_uv, dtype=np.int32).reshape(-1, 2)
    H, W = cL.shape
    out = np.zeros(len(q), np.int32)
    lib().or_epipolar_match(_p(cL), _p(cR), W, H, _p(q), len(q), int(dmax), int(t_lo), int(margin), _p(out))
    return out


def incircle_sos(P, a, b, c, d):
    P = np.ascontiguousarray(P, dtype=np.int32).reshape(-1, 2)
    return lib().or_incircle_sos(_p(P), int(a), int(b), int(c), int(d))


def delaunay(P):
    """Triangles (T, 3) of sorted index triples for points P (n, 2) in canonical order."""
    P = np.ascontiguousarray(P, dtype=np.int32).reshape(-1, 2)
    n = len(P)
    cap = 2 * n + 16
    out = np.zeros((cap, 3), np.int32)
    T = lib().or_delaunay(_p(P), n, _p(out), cap)
    if T < 0:
        raise RuntimeError(f"or_delaunay failed: {T}")
    return out[:T].copy()


def planes(P, D, tri):
    P = np.ascontiguousarray(P, dtype=np.int32).reshape(-1, 2)
    D = np.ascontiguousarray(D, dtype=np.float32)
    tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((len(tri), 3), np.float32)
    lib().or_planes(_p(P), _p(D), _p(tri), len(tri), _p(out))
    return out


def raster(P, tri, W, H):
    P = np.ascontiguousarray(P, dtype=np.int32).reshape(-1, 2)
    tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((H, W), np.int32)
    rc = lib().or_raster(_p(P), _p(tri), len(tri), W, H, _p(out))
    if rc != 0:
        raise RuntimeError(f"or_raster failed: {rc}")
    return out


def interp_map(planeidx, abc):
    """DisparityInterpolation: D_it over the lookup table (NaN without a triangle)."""
    planeidx = np.ascontiguousarray(planeidx, dtype=np.int32)
    H, W = planeidx.shape
    out = np.zeros((H, W), np.float32)
    lib().or_interp_map(_p(planeidx), _p(np.ascontiguousarray(abc, dtype=np.float32)), W, H, _p(out))
    return out


def validate(cL, cR, om, planeidx, abc, sz, Df, Cf, t_lo=DEFAULT_PARAMS["t_lo"], t_hi=DEFAULT_PARAMS["t_hi"]):
    """One CostEvaluation + DisparityRefinement pass.  Df, Cf are updated in place.
    Returns mask and the cell records as a dict."""
    H, W = cL.shape
    Wc, Hc = -(-W // sz), -(-H // sz)
    nc = Wc * Hc
    mask = np.zeros((H, W), np.uint8)
    r = dict(cg_uv=np.zeros((nc, 2), np.int32), cg_d=np.zeros(nc, np.float32), cg_cost=np.zeros(nc, np.int32),
             cg_w=np.zeros(nc, np.uint8), cb_uv=np.zeros((nc, 2), np.int32), cb_cost=np.zeros(nc, np.int32),
             cb_w=np.zeros(nc, np.uint8))
    lib().or_validate(_p(np.ascontiguousarray(cL)), _p(np.ascontiguousarray(cR)), _p(np.ascontiguousarray(om)),
                      _p(np.ascontiguousarray(planeidx, dtype=np.int32)), _p(np.ascontiguousarray(abc, dtype=np.float32)),
                      W, H, int(sz), int(t_lo), int(t_hi), _p(Df), _p(Cf), _p(mask),
                      _p(r["cg_uv"]), _p(r["cg_d"]), _p(r["cg_cost"]), _p(r["cg_w"]),
                      _p(r["cb_uv"]), _p(r["cb_cost"]), _p(r["cb_w"]))
    r["mask"] = mask
    r["Wc"], r["Hc"] = Wc, Hc
    return r


class _Sp(ctypes.Structure):
    _fields_ = [("u", ctypes.c_int32), ("v", ctypes.c_int32), ("d", ctypes.c_float)]


def resample(cL, cR, sz, cells, S, dmax, t_lo=DEFAULT_PARAMS["t_lo"], margin=DEFAULT_PARAMS["uniq_margin"]):
    """SupportResampling.  S: structured (n, 3) float array (u, v, d); returns the new set."""
    H, W = cL.shape
    S = np.asarray(S, dtype=np.float64).reshape(-1, 3)
    cap = W * H
    buf = np.zeros(cap, dtype=np.dtype([("u", np.int32), ("v", np.int32), ("d", np.float32)]))
    buf["u"][:len(S)] = S[:, 0]
    buf["v"][:len(S)] = S[:, 1]
    buf["d"][:len(S)] = S[:, 2]
    n = lib().or_resample(_p(np.ascontiguousarray(cL)), _p(np.ascontiguousarray(cR)), W, H, int(sz),
                          _p(cells["cg_uv"]), _p(cells["cg_d"]), _p(cells["cg_w"]),
                          _p(cells["cb_uv"]), _p(cells["cb_w"]), int(dmax), int(t_lo), int(margin),
                          _p(buf), len(S), cap)
    if n < 0:
        raise RuntimeError(f"or_resample failed: {n}")
    out = buf[:n]
    return np.stack([out["u"].astype(np.float64), out["v"].astype(np.float64), out["d"].astype(np.float64)], 1)


def run(left, right, dmax, iters, cell, **params):
    """The whole method (Alg. 1) for one pair.  Returns a dict with D_f, C_f, mask,
    planeidx (last pass), and the per-iteration support sets and triangle counts."""
    prm = dict(DEFAULT_PARAMS)
    prm.update(params)
    L = np.ascontiguousarray(left, dtype=np.uint8)
    R = np.ascontiguousarray(right, dtype=np.uint8)
    H, W = L.shape
    Df = np.zeros((H, W), np.float32)
    Cf = np.zeros((H, W), np.uint8)
    mask = np.zeros((H, W), np.uint8)
    pidx = np.zeros((H, W), np.int32)
    cap = 3 * W * H * iters + 3000
    trace = np.zeros(cap, np.float32)
    ns = np.zeros(iters, np.int32)
    nt = np.zeros(iters, np.int32)
    P = _Params(**prm)
    rc = lib().or_run(_p(L), _p(R), W, H, int(dmax), int(iters), int(cell), ctypes.byref(P),
                      _p(Df), _p(Cf), _p(mask), _p(pidx), _p(trace), cap, _p(ns), _p(nt))
    if rc != 0:
        raise RuntimeError(f"or_run failed: {rc}")
    sup, pos = [], 0
    for it in range(iters):
        k = int(ns[it])
        sup.append(trace[pos:pos + 3 * k].reshape(k, 3).copy())
        pos += 3 * k
    return dict(D_f=Df, C_f=Cf, mask=mask, planeidx=pidx, support=sup, n_tri=nt.copy())
