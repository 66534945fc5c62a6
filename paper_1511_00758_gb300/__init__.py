"""Python binding of libstereo (include/stereo.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module loads it with
ctypes, converts tensors and arrays to pointers, and raises StereoError on a
negative return code.  There is no Python or CPU fallback: if the library is
missing or cannot load, import-time calls raise.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

__all__ = [
    "StereoError", "load", "lib", "Config", "Result", "Pair", "Stats", "Tuning", "Context", "request_bytes",
    "census", "fast", "epipolar_match", "delaunay", "delaunay_parallel", "delaunay_insert", "planes", "raster_scratch_bytes", "raster", "raster_noalloc", "validate_bulk",
    "validate", "resample_match", "ERRORS",
]

ERRORS = {0: "OK", -1: "INVAL", -2: "NOMEM", -3: "BUSY", -4: "PENDING", -5: "TIMEOUT",
          -6: "INTERNAL", -7: "CUDA", -8: "NOTFOUND", -9: "CAP"}
E_PENDING = -4


class StereoError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"libstereo {what}: {ERRORS.get(code, code)} ({code})")


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("mem_budget_bytes", ctypes.c_size_t), ("arena", ctypes.c_void_p),
                ("max_slots", ctypes.c_int), ("max_queue", ctypes.c_int), ("t_lo", ctypes.c_int),
                ("t_hi", ctypes.c_int), ("t_grad", ctypes.c_int), ("t_fast", ctypes.c_int),
                ("kp_per_bin", ctypes.c_int), ("uniq_margin", ctypes.c_int), ("host_threads", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("profile", ctypes.c_int), ("inject_mesh_failure", ctypes.c_int),
                ("batch_window_us", ctypes.c_int), ("autotune", ctypes.c_int), ("tune_w", ctypes.c_int),
                ("tune_h", ctypes.c_int), ("host_mesh", ctypes.c_int), ("inject_wait_timeout", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("disparity", ctypes.c_void_p), ("cost", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("planeidx", ctypes.c_void_p), ("w", ctypes.c_int), ("h", ctypes.c_int), ("iters", ctypes.c_int),
                ("n_support", ctypes.POINTER(ctypes.c_int32)), ("n_tri", ctypes.POINTER(ctypes.c_int32)),
                ("support", ctypes.POINTER(ctypes.c_float)), ("latency_ms", ctypes.c_double),
                ("host_mesh_ms", ctypes.c_double), ("status", ctypes.c_int)]


class Pair(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_int), ("left", ctypes.c_void_p), ("right", ctypes.c_void_p),
                ("w", ctypes.c_int), ("h", ctypes.c_int), ("dmax", ctypes.c_int), ("iters", ctypes.c_int),
                ("cell", ctypes.c_int), ("out_disparity", ctypes.c_void_p), ("out_cost", ctypes.c_void_p),
                ("out_mask", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("requests_done", ctypes.c_longlong),
                ("batched_pairs", ctypes.c_longlong), ("gpu_rounds", ctypes.c_longlong),
                ("host_mesh_ms", ctypes.c_double), ("kind_launches", ctypes.c_longlong * 10),
                ("kind_ms", ctypes.c_double * 10), ("kind_bytes", ctypes.c_double * 10),
                ("round_ms", ctypes.c_double), ("graph_ms", ctypes.c_double), ("exec_ms", ctypes.c_double),
                ("graph_instantiations", ctypes.c_longlong), ("kind_timed", ctypes.c_longlong * 10),
                ("mesh_passes", ctypes.c_longlong), ("mesh_insert_rounds", ctypes.c_longlong),
                ("mesh_flip_rounds", ctypes.c_longlong), ("mesh_flips", ctypes.c_longlong),
                ("mesh_points", ctypes.c_longlong), ("mesh_edge_points", ctypes.c_longlong)]


class Tuning(ctypes.Structure):
    _fields_ = [("small_area", ctypes.c_int), ("batch_area", ctypes.c_int), ("raster_cols", ctypes.c_int),
                ("validate_blocks_per_sm", ctypes.c_int), ("validate_mixed", ctypes.c_int), ("autotuned", ctypes.c_int),
                ("raster_us", ctypes.c_double), ("validate_us", ctypes.c_double)]


KINDS = ("census", "fast_score", "fast_bins", "match_kp", "raster_clear", "raster", "validate", "resample", "fill",
         "mesh")


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "stereo_default_config": (None, [ctypes.POINTER(Config)]),
    "stereo_create": (_I, [ctypes.POINTER(Config), ctypes.POINTER(_P)]),
    "stereo_submit": (_I, [_P, _I, _P, _P, _I, _I, _I, _I, _I, ctypes.POINTER(ctypes.c_uint64)]),
    "stereo_submit_batch": (_I, [_P, ctypes.POINTER(Pair), _I, ctypes.POINTER(ctypes.c_uint64)]),
    "stereo_request_bytes": (ctypes.c_size_t, [ctypes.POINTER(Config), _I, _I, _I, _I, _I]),
    "stereo_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(Result), _I]),
    "stereo_poll_host": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(Result), _I, _P, _P, _P]),
    "stereo_release": (_I, [_P, ctypes.c_uint64]),
    "stereo_poll_batch": (_I, [_P, ctypes.POINTER(ctypes.c_uint64), _I, ctypes.POINTER(Result), _I]),
    "stereo_release_batch": (_I, [_P, ctypes.POINTER(ctypes.c_uint64), _I]),
    "stereo_destroy": (None, [_P]),
    "stereo_get_stats": (_I, [_P, ctypes.POINTER(Stats)]),
    "stereo_get_tuning": (_I, [_P, ctypes.POINTER(Tuning)]),
    "stereo_last_error": (ctypes.c_char_p, []),
    "stereo_census": (_I, [_P, _P, _I, _I, _I, _P, _P, _P, _P]),
    "stereo_fast": (_I, [_P, _I, _I, _I, _I, _P, _P, _P]),
    "stereo_epipolar_match": (_I, [_P, _P, _I, _I, _P, _I, _I, _I, _I, _P, _P]),
    "stereo_delaunay": (_I, [_P, _I, _P, _I]),
    "stereo_delaunay_parallel": (_I, [_P, _I, _P, _I, _I]),
    "stereo_delaunay_insert": (_I, [_P, _I, _P, _I, _P, _I, _I, _I, _P, _I]),
    "stereo_planes": (_I, [_P, _P, _P, _I, _P]),
    "stereo_raster_scratch_bytes": (ctypes.c_size_t, [_I]),
    "stereo_raster": (_I, [_P, _P, _I, _I, _I, _P, _P, _P, ctypes.c_size_t, _P]),
    "stereo_raster_noalloc": (_I, [_P, _P, _I, _I, _I, _P, _P, _P]),
    "stereo_validate": (_I, [_P, _P, _P, _P, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P]),
    "stereo_validate_bulk": (_I, [_P, _P, _P, _P, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P]),
    "stereo_resample_match": (_I, [_P, _P, _I, _P, _P, _P, _I, _I, _I, _I, _I, _P, _P, _P]),
}
SYMBOLS = tuple(_SIGS)


def load(path=None, build=True):
    """Load libstereo.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise StereoError(-7, f"library missing at {path}")
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def lib():
    return _lib if _lib is not None else load()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc, what):
    if rc < 0:
        if rc in (-6, -7) and _lib is not None:
            what = f"{what} [{_lib.stereo_last_error().decode()}]"
        raise StereoError(rc, what)
    return rc


def request_bytes(w, h, dmax, iters, cell, host_mesh=0, kp_per_bin=4):
    """Device memory one request of this shape takes from a context's budget."""
    cfg = Config()
    lib().stereo_default_config(ctypes.byref(cfg))
    cfg.host_mesh = host_mesh
    cfg.kp_per_bin = kp_per_bin
    return int(lib().stereo_request_bytes(ctypes.byref(cfg), w, h, dmax, iters, cell))


# ---------------------------------------------------------------- stage calls
def census(left, right, w, h, t_grad, cL, cR, omega, stream=None):
    return _check(lib().stereo_census(_ptr(left), _ptr(right), w, h, t_grad, _ptr(cL), _ptr(cR), _ptr(omega),
                                      _stream(stream)), "census")


def fast(left, w, h, t_fast, K, scratch, out_uv, stream=None):
    return _check(lib().stereo_fast(_ptr(left), w, h, t_fast, K, _ptr(scratch), _ptr(out_uv), _stream(stream)),
                  "fast")


def epipolar_match(cL, cR, w, h, q_uv, n, dmax, t_lo, margin, out_d, stream=None):
    return _check(lib().stereo_epipolar_match(_ptr(cL), _ptr(cR), w, h, _ptr(q_uv), n, dmax, t_lo, margin,
                                              _ptr(out_d), _stream(stream)), "epipolar_match")


def delaunay(uv, n, tri, cap):
    """Host call: uv, tri are host (numpy) buffers.  Returns the triangle count."""
    return _check(lib().stereo_delaunay(_ptr(uv), n, _ptr(tri), cap), "delaunay")


def delaunay_parallel(uv, n, tri, cap, threads):
    """Host call, as delaunay, with the top splits on up to `threads` host threads."""
    return _check(lib().stereo_delaunay_parallel(_ptr(uv), n, _ptr(tri), cap, threads), "delaunay_parallel")


def delaunay_insert(uv, n, tri, T, uv_new, m, w, h, tri_out, cap):
    """Device re-tessellation: the triangulation of uv + uv_new by insertion into (uv, tri) (host arrays)."""
    return _check(lib().stereo_delaunay_insert(_ptr(uv), n, _ptr(tri), T, _ptr(uv_new), m, w, h, _ptr(tri_out), cap),
                  "delaunay_insert")


def planes(uv, d, tri, T, abc):
    return _check(lib().stereo_planes(_ptr(uv), _ptr(d), _ptr(tri), T, _ptr(abc)), "planes")


def raster_scratch_bytes(T):
    return int(lib().stereo_raster_scratch_bytes(T))


def raster(tri_uv, abc, T, w, h, planeidx, D_it, scratch, scratch_bytes, stream=None):
    return _check(lib().stereo_raster(_ptr(tri_uv), _ptr(abc), T, w, h, _ptr(planeidx), _ptr(D_it), _ptr(scratch),
                                      scratch_bytes, _stream(stream)), "raster")


def raster_noalloc(tri_uv, abc, T, w, h, planeidx, D_it, stream=None):
    """stereo_raster with its work lists in the library's fixed device array
    (for callers that cannot allocate device memory); T <= 262143."""
    return _check(lib().stereo_raster_noalloc(_ptr(tri_uv), _ptr(abc), T, w, h, _ptr(planeidx), _ptr(D_it),
                                              _stream(stream)), "raster_noalloc")


def validate(cL, cR, omega, D_it, w, h, sz, t_lo, t_hi, first_pass, D_f, C_f, mask, cg_key, cb_key, stream=None):
    return _check(lib().stereo_validate(_ptr(cL), _ptr(cR), _ptr(omega), _ptr(D_it), w, h, sz, t_lo, t_hi,
                                        int(first_pass), _ptr(D_f), _ptr(C_f), _ptr(mask), _ptr(cg_key),
                                        _ptr(cb_key), _stream(stream)), "validate")


def validate_bulk(cL, cR, omega, D_it, w, h, sz, t_lo, t_hi, first_pass, D_f, C_f, mask, cg_key, cb_key, err_flag,
                  stream=None):
    return _check(lib().stereo_validate_bulk(_ptr(cL), _ptr(cR), _ptr(omega), _ptr(D_it), w, h, sz, t_lo, t_hi,
                                             int(first_pass), _ptr(D_f), _ptr(C_f), _ptr(mask), _ptr(cg_key),
                                             _ptr(cb_key), _ptr(err_flag), _stream(stream)), "validate_bulk")


def resample_match(cg_key, cb_key, ncells, D_it, cL, cR, w, h, dmax, t_lo, margin, cg_d, x_d, stream=None):
    return _check(lib().stereo_resample_match(_ptr(cg_key), _ptr(cb_key), ncells, _ptr(D_it), _ptr(cL), _ptr(cR),
                                              w, h, dmax, t_lo, margin, _ptr(cg_d), _ptr(x_d), _stream(stream)),
                  "resample_match")


# ---------------------------------------------------------------- request API
class Context:
    """stereo_create / submit / poll / release / destroy.  Device memory for
    in-flight requests is one arena tensor from the PyTorch caching allocator;
    the library sub-allocates it.  The stream is a torch stream."""

    def __init__(self, device=0, mem_budget_bytes=1 << 30, max_slots=1, max_queue=64, host_threads=1,
                 stream=None, **params):
        import torch
        L = lib()
        cfg = Config()
        L.stereo_default_config(ctypes.byref(cfg))
        cfg.device = device
        cfg.max_slots = max_slots
        cfg.max_queue = max_queue
        cfg.host_threads = host_threads
        for k, v in params.items():
            if not hasattr(cfg, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(cfg, k, v)
        self.arena = torch.empty(mem_budget_bytes, dtype=torch.uint8, device=f"cuda:{device}")
        cfg.arena = self.arena.data_ptr()
        cfg.mem_budget_bytes = mem_budget_bytes
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        cfg.stream = self.stream.cuda_stream
        self.cfg = cfg
        h = _P()
        _check(L.stereo_create(ctypes.byref(cfg), ctypes.byref(h)), "create")
        self.h = h

    def submit(self, left, right, w, h, dmax, iters, cell, stream_id=0):
        t = ctypes.c_uint64()
        _check(lib().stereo_submit(self.h, stream_id, _ptr(left), _ptr(right), w, h, dmax, iters, cell,
                                   ctypes.byref(t)), "submit")
        return t.value

    def submit_batch(self, pairs):
        """pairs: (left, right, w, h, dmax, iters, cell[, stream_id[, outputs]]) tuples, where
        outputs is (disparity, cost, mask) (each a buffer or None) that receives D_f, C_f and
        the mask before the request is done.  Returns the tickets of the pairs taken (a
        prefix of the list; raises when none is)."""
        arr = (Pair * len(pairs))()
        for i, q in enumerate(pairs):
            left, right, w, h, dmax, iters, cell = q[:7]
            out = q[8] if len(q) > 8 and q[8] is not None else (None, None, None)
            arr[i] = Pair(q[7] if len(q) > 7 else 0, _ptr(left), _ptr(right), w, h, dmax, iters, cell,
                          _ptr(out[0]), _ptr(out[1]), _ptr(out[2]))
        tk = (ctypes.c_uint64 * len(pairs))()
        n = _check(lib().stereo_submit_batch(self.h, arr, len(pairs), tk), "submit_batch")
        return list(tk[:n])

    def poll(self, ticket, timeout_us=-1):
        r = Result()
        rc = lib().stereo_poll(self.h, ticket, ctypes.byref(r), timeout_us)
        if rc == E_PENDING:
            return None
        _check(rc, "poll")
        return r

    def poll_host(self, ticket, disparity, cost, mask=None, timeout_us=-1):
        """poll, then D_f / C_f / mask copied by the library into the given host
        buffers (numpy arrays or CPU tensors; page-locked copies fastest)."""
        r = Result()
        rc = lib().stereo_poll_host(self.h, ticket, ctypes.byref(r), timeout_us, _ptr(disparity), _ptr(cost),
                                    _ptr(mask))
        if rc == E_PENDING:
            return None
        _check(rc, "poll_host")
        return r

    def release(self, ticket):
        return _check(lib().stereo_release(self.h, ticket), "release")

    def poll_batch(self, tickets, timeout_us=-1):
        """poll for every ticket at once: the list of results (each with its own status) once
        all are done, or None when the time ran out first."""
        tk = (ctypes.c_uint64 * len(tickets))(*tickets)
        out = (Result * len(tickets))()
        rc = lib().stereo_poll_batch(self.h, tk, len(tickets), out, timeout_us)
        if rc == E_PENDING:
            return None
        _check(rc, "poll_batch")
        return list(out)

    def release_batch(self, tickets):
        tk = (ctypes.c_uint64 * len(tickets))(*tickets)
        return _check(lib().stereo_release_batch(self.h, tk, len(tickets)), "release_batch")

    def stats(self):
        s = Stats()
        _check(lib().stereo_get_stats(self.h, ctypes.byref(s)), "stats")
        return s

    def tuning(self):
        """The kernels' work shapes in use, as a dict (see stereo_get_tuning)."""
        t = Tuning()
        _check(lib().stereo_get_tuning(self.h, ctypes.byref(t)), "tuning")
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().stereo_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def result_tensors(self, r):
        """Copies of a polled result's device buffers as torch tensors, plus the trace."""
        import numpy as np
        import torch
        H, W = r.h, r.w
        with torch.cuda.stream(self.stream):
            out = dict(D_f=device_view(r.disparity, (H, W), "<f4").clone(),
                       C_f=device_view(r.cost, (H, W), "|u1").clone(),
                       mask=device_view(r.mask, (H, W), "|u1").clone(),
                       planeidx=device_view(r.planeidx, (H, W), "<i4").clone())
        self.stream.synchronize()
        ns = [r.n_support[i] for i in range(r.iters)]
        nt = [r.n_tri[i] for i in range(r.iters)]
        tot = 3 * sum(ns)
        flat = np.ctypeslib.as_array(r.support, shape=(tot,)).copy() if tot else np.zeros(0, np.float32)
        sup, pos = [], 0
        for k in ns:
            sup.append(flat[pos:pos + 3 * k].reshape(k, 3))
            pos += 3 * k
        out.update(support=sup, n_tri=nt, latency_ms=r.latency_ms, host_mesh_ms=r.host_mesh_ms)
        return out


class _DevArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_view(ptr, shape, typestr):
    """Zero-copy torch view of library-owned device memory (valid until release)."""
    import torch
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")
