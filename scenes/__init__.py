"""Seeded synthetic rectified stereo pairs of piecewise-planar scenes.

These inputs stand in for the KITTI, Bumblebee2 and ZED imagery of the paper's
experiments (Sec. IV), which are not available here.  A scene is a stack of
planar surfaces, each with a disparity plane d = a*u + b*v + c in left-image
coordinates (Eq. 3) and a convex polygonal footprint, textured with 4-octave
value noise that sticks to the surface.  The left image shows the front-most
(largest-d) surface at every pixel; the right image is rendered by solving for
the left source column u of every right pixel x (x = u - d(u, v)) per surface
and again keeping the front-most one, so occlusions are filled by whatever is
visible behind.  Ground-truth disparity is the front surface's plane, exactly.

This module holds no arithmetic of the stereo method itself; it only makes
inputs.  Both the CPU oracle tests and the CUDA path draw from it.
"""
from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

__all__ = [
    "Surface", "Scene", "StereoPair", "polygon_scene", "driving_scene",
    "render", "make_pair", "CONFIGS", "config_pairs", "integer_shift_pair", "mixed_pairs", "serving_streams",
    "large_pairs", "burst_pairs", "sweep_pairs", "SWEEP_SIZES",
]

_OCT_SPACING = (16.0, 8.0, 4.0, 2.0)
_OCT_AMP = (1.0, 0.5, 0.25, 0.125)


@dataclasses.dataclass
class Surface:
    a: float
    b: float
    c: float
    poly: np.ndarray | None   # (n, 2) convex polygon (u, v), counter-clockwise in (u, v); None = everywhere
    salt: int                 # texture hash salt
    tex_off: tuple            # texture offset (ou, ov)


@dataclasses.dataclass
class Scene:
    width: int
    height: int
    surfaces: list
    sigma: float
    unmatched_frac: float
    noise_seed: int


@dataclasses.dataclass
class StereoPair:
    left: np.ndarray      # uint8 [H, W]
    right: np.ndarray     # uint8 [H, W]
    gt_disp: np.ndarray   # float32 [H, W], left-view disparity of the front surface
    gt_occ: np.ndarray    # bool [H, W], left pixel not visible in the right image
    dmax: int
    iters: int
    cell: int


def _hash(ix, iy, salt):
    """32-bit integer hash of lattice coordinates (murmur3 finaliser)."""
    with np.errstate(over="ignore"):
        h = (ix.astype(np.uint32) * np.uint32(0x8DA6B343)) ^ (iy.astype(np.uint32) * np.uint32(0xD8163841))
        h ^= np.uint32(salt & 0xFFFFFFFF)
        h ^= h >> np.uint32(16)
        h *= np.uint32(0x85EBCA6B)
        h ^= h >> np.uint32(13)
        h *= np.uint32(0xC2B2AE35)
        h ^= h >> np.uint32(16)
    return h


def value_noise(x, y, salt):
    """4-octave value noise in [0, 255] at real coordinates (x, y)."""
    total = np.zeros(np.broadcast(x, y).shape, dtype=np.float64)
    for o, (sp, amp) in enumerate(zip(_OCT_SPACING, _OCT_AMP)):
        fx = x / sp
        fy = y / sp
        ix = np.floor(fx)
        iy = np.floor(fy)
        tx = fx - ix
        ty = fy - iy
        sx = tx * tx * (3.0 - 2.0 * tx)
        sy = ty * ty * (3.0 - 2.0 * ty)
        ix = ix.astype(np.int64)
        iy = iy.astype(np.int64)
        s = salt * 8 + o
        v00 = _hash(ix, iy, s).astype(np.float64)
        v10 = _hash(ix + 1, iy, s).astype(np.float64)
        v01 = _hash(ix, iy + 1, s).astype(np.float64)
        v11 = _hash(ix + 1, iy + 1, s).astype(np.float64)
        top = v00 + (v10 - v00) * sx
        bot = v01 + (v11 - v01) * sx
        total += amp * (top + (bot - top) * sy) / 4294967296.0
    return total * (255.0 / sum(_OCT_AMP))


def _inside_convex(poly, px, py):
    """Point-in-convex-polygon (closed) for a CCW polygon in (u, v)."""
    inside = np.ones(np.broadcast(px, py).shape, dtype=bool)
    n = len(poly)
    for i in range(n):
        x0, y0 = poly[i]
        x1, y1 = poly[(i + 1) % n]
        cross = (x1 - x0) * (py - y0) - (y1 - y0) * (px - x0)
        inside &= cross >= 0.0
    return inside


def render(scene: Scene):
    """Render (left, right, gt_disp, gt_occ) for a scene."""
    W, H = scene.width, scene.height
    uu, vv = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    # left view: front-most surface at each pixel
    best_d = np.full((H, W), -np.inf)
    best_s = np.full((H, W), -1, dtype=np.int64)

    def window(s, right):
        """Row/column slices that can contain the surface (the whole image without a polygon)."""
        if s.poly is None:
            return slice(0, H), slice(0, W)
        u0, u1 = s.poly[:, 0].min(), s.poly[:, 0].max()
        v0, v1 = s.poly[:, 1].min(), s.poly[:, 1].max()
        if right:  # x = u - d(u, v); d is linear, so its extremes sit at the vertices
            dv = s.a * s.poly[:, 0] + s.b * s.poly[:, 1] + s.c
            u0, u1 = u0 - dv.max(), u1 - dv.min()
        r = slice(int(np.clip(np.floor(v0) - 1, 0, H)), int(np.clip(np.ceil(v1) + 2, 0, H)))
        c = slice(int(np.clip(np.floor(u0) - 1, 0, W)), int(np.clip(np.ceil(u1) + 2, 0, W)))
        return r, c

    for si, s in enumerate(scene.surfaces):
        r, c = window(s, False)
        U, V = uu[r, c], vv[r, c]
        d = s.a * U + s.b * V + s.c
        bd = best_d[r, c]
        m = d > bd
        if s.poly is not None:
            m &= _inside_convex(s.poly, U, V)
        bd[m] = d[m]
        best_s[r, c][m] = si
    # right view: for right pixel x, source column u solves u - d(u, v) = x
    rbest_d = np.full((H, W), -np.inf)
    rbest_s = np.full((H, W), -1, dtype=np.int64)
    rsrc_u = np.zeros((H, W))
    for si, s in enumerate(scene.surfaces):
        r, c = window(s, True)
        X, V = uu[r, c], vv[r, c]
        u_src = (X + s.b * V + s.c) / (1.0 - s.a)
        d = u_src - X
        bd = rbest_d[r, c]
        m = d > bd
        if s.poly is not None:
            m &= _inside_convex(s.poly, u_src, V)
        bd[m] = d[m]
        rbest_s[r, c][m] = si
        rsrc_u[r, c][m] = u_src[m]
    assert (best_s >= 0).all() and (rbest_s >= 0).all(), "scene must cover the image (background surface)"
    left_f = np.zeros((H, W))
    right_f = np.zeros((H, W))
    for si, s in enumerate(scene.surfaces):
        ml = best_s == si
        if ml.any():
            left_f[ml] = value_noise(uu[ml] + s.tex_off[0], vv[ml] + s.tex_off[1], s.salt)
        mr = rbest_s == si
        if mr.any():
            right_f[mr] = value_noise(rsrc_u[mr] + s.tex_off[0], vv[mr] + s.tex_off[1], s.salt)
    rng = np.random.Generator(np.random.PCG64(scene.noise_seed))
    if scene.sigma > 0:
        left_f += rng.standard_normal((H, W)) * scene.sigma
        right_f += rng.standard_normal((H, W)) * scene.sigma
    left = np.clip(np.rint(left_f), 0, 255).astype(np.uint8)
    right = np.clip(np.rint(right_f), 0, 255).astype(np.uint8)
    if scene.unmatched_frac > 0:
        m = rng.random((H, W)) < scene.unmatched_frac
        right[m] = rng.integers(0, 256, size=int(m.sum()), dtype=np.uint8)
    # occlusion: left pixel whose right-image location shows a nearer surface
    xr = np.rint(uu - best_d).astype(np.int64)
    outside = (xr < 0) | (xr >= W)
    xr_c = np.clip(xr, 0, W - 1)
    rows = np.arange(H)[:, None].repeat(W, 1)
    occ = outside | (rbest_d[rows, xr_c] > best_d + 0.5)
    return left, right, best_d.astype(np.float32), occ


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _background(rng, W, H, dlo, dhi):
    a = rng.uniform(-0.004, 0.004)
    b = rng.uniform(-0.004, 0.004)
    corners = [a * u + b * v for u in (0, W - 1) for v in (0, H - 1)]
    lo, hi = min(corners), max(corners)
    c = rng.uniform(dlo - lo, max(dlo - lo, dhi - hi - 1e-3))
    return a, b, c


def _plane_over(rng, pts, dlo, dhi, slope):
    """Plane with |a|,|b| <= slope whose values over pts lie in [dlo, dhi)."""
    for _ in range(100):
        a = rng.uniform(-slope, slope)
        b = rng.uniform(-slope, slope)
        lin = a * pts[:, 0] + b * pts[:, 1]
        lo, hi = dlo - lin.min(), dhi - 1e-3 - lin.max()
        if hi > lo:
            return a, b, rng.uniform(lo, hi)
    return 0.0, 0.0, rng.uniform(dlo, dhi - 1e-3)


def polygon_scene(W, H, seed, n_poly=20, dmax=64, sigma=2.0, unmatched=0.0, slope=0.05):
    """Background plane (d in [0, 8)) plus random convex planar polygons with d in [0, dmax)."""
    rng = _rng(seed)
    surfs = []
    a, b, c = _background(rng, W, H, 0.0, 8.0)
    surfs.append(Surface(a, b, c, None, int(rng.integers(1, 2**31)), tuple(rng.uniform(1000, 50000, 2))))
    rscale = max(1.0, min(W / 640.0, H / 480.0))
    for _ in range(n_poly):
        cu, cv = rng.uniform(0, W), rng.uniform(0, H)
        r = rng.uniform(20, 150) * rscale
        nv = int(rng.integers(3, 9))
        ang = np.sort(rng.uniform(0, 2 * math.pi, nv))
        poly = np.stack([cu + r * np.cos(ang), cv + r * np.sin(ang)], 1)
        a, b, c = _plane_over(rng, poly, 0.0, float(dmax), slope)
        surfs.append(Surface(a, b, c, poly, int(rng.integers(1, 2**31)), tuple(rng.uniform(1000, 50000, 2))))
    return Scene(W, H, surfs, sigma, unmatched, int(rng.integers(1, 2**62)))


def driving_scene(W, H, seed, n_box=40, dmax=128, ground_max=96.0, sigma=3.0, unmatched=0.05, slope=0.05):
    """Far wall, a ground plane with d linear in v (0 at the horizon row H/3, ground_max at the
    bottom row) and fronto-parallel or slanted rectangular boxes with d in [0, dmax)."""
    rng = _rng(seed)
    surfs = []
    surfs.append(Surface(0.0, 0.0, rng.uniform(0.0, 1.0), None, int(rng.integers(1, 2**31)),
                         tuple(rng.uniform(1000, 50000, 2))))
    h0 = H / 3.0
    gb = ground_max / (H - 1 - h0)
    big = 1e7
    ground = np.array([[-big, h0], [big, h0], [big, big], [-big, big]])
    # CCW in (u, v) means positive cross for the interior: check orientation below
    surfs.append(Surface(0.0, gb, -gb * h0, _ccw(ground), int(rng.integers(1, 2**31)),
                         tuple(rng.uniform(1000, 50000, 2))))
    for _ in range(n_box):
        w = rng.uniform(20, 200)
        h = rng.uniform(20, 150)
        u0 = rng.uniform(-w / 2, W - w / 2)
        v0 = rng.uniform(h0 - h, H - h / 2)
        poly = np.array([[u0, v0], [u0 + w, v0], [u0 + w, v0 + h], [u0, v0 + h]])
        if rng.random() < 0.5:
            a, b, c = 0.0, 0.0, rng.uniform(4.0, dmax - 4.0)
        else:
            a, b, c = _plane_over(rng, poly, 0.0, float(dmax), slope)
        surfs.append(Surface(a, b, c, _ccw(poly), int(rng.integers(1, 2**31)),
                             tuple(rng.uniform(1000, 50000, 2))))
    return Scene(W, H, surfs, sigma, unmatched, int(rng.integers(1, 2**62)))


def _ccw(poly):
    """Order a convex polygon so that the interior has a positive edge cross product."""
    x, y = poly[:, 0], poly[:, 1]
    area2 = np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)
    return poly if area2 > 0 else poly[::-1].copy()


def make_pair(kind, W, H, seed, dmax, iters, cell, **kw):
    if kind == "polygon":
        sc = polygon_scene(W, H, seed, dmax=dmax, **kw)
    elif kind == "driving":
        sc = driving_scene(W, H, seed, dmax=dmax, **kw)
    else:
        raise ValueError(kind)
    for s in sc.surfaces:
        if s.poly is not None:
            s.poly = _ccw(s.poly)
    left, right, gt, occ = render(sc)
    return StereoPair(left, right, gt, occ, dmax, iters, cell)


SEED_BASE = 0x5EED0000

# The five workloads: (description, list of pair specs).  A pair spec is
# (kind, W, H, dmax, iters, cell, extra kwargs).
CONFIGS = {
    "vga_polygons": dict(kind="polygon", W=640, H=480, dmax=64, iters=1, cell=16, n=1, idx=0,
                         kw=dict(n_poly=20, sigma=2.0)),
    "driving_1242x375": dict(kind="driving", W=1242, H=375, dmax=128, iters=3, cell=8, n=1, idx=1,
                             kw=dict(n_box=40, sigma=3.0, unmatched=0.05)),
}


def _mixed_spec(i):
    """Pair i of the uneven batch: 16 each of 320x240, 640x480, 1242x375 (driving), 1280x720;
    dmax drawn from 64..128 per pair; 3 iterations, 16x16 cells."""
    sizes = [(320, 240, "polygon"), (640, 480, "polygon"), (1242, 375, "driving"), (1280, 720, "polygon")]
    W, H, kind = sizes[i % 4]
    dmax = int(_rng(SEED_BASE + 2000 + 7919 * i).integers(64, 129))
    return kind, W, H, dmax


def mixed_pairs(n=64, cache_dir=None):
    """The uneven batch (64 pairs of four sizes, mixed dmax)."""
    out = []
    for i in range(n):
        kind, W, H, dmax = _mixed_spec(i)
        kw = dict(n_box=40, sigma=3.0, unmatched=0.05) if kind == "driving" else dict(n_poly=20, sigma=2.0)
        out.append(_cached(f"mixed_{i}", cache_dir, lambda: make_pair(kind, W, H, SEED_BASE + 2000 + i, dmax, 3, 16, **kw),
                           dmax, 3, 16))
    return out


def serving_streams(cache_dir=None):
    """Eight camera streams: four 640x480 (dmax 64) and four 1280x720 (dmax 128); one rendered pair
    per stream (frames of a stream are the same seeded scene); 2 iterations, 16x16 cells."""
    out = []
    for i in range(8):
        W, H, dmax = (640, 480, 64) if i < 4 else (1280, 720, 128)
        out.append(_cached(f"serving_{i}", cache_dir,
                           lambda: make_pair("polygon", W, H, SEED_BASE + 3000 + i, dmax, 2, 16, n_poly=20, sigma=2.0),
                           dmax, 2, 16))
    return out


def large_pairs(n=16, cache_dir=None):
    """2048x1536 pairs, 30-plane scenes, dmax 256, 5 iterations, 4x4 initial cells."""
    return [_cached(f"large_{i}", cache_dir,
                    lambda: make_pair("polygon", 2048, 1536, SEED_BASE + 4000 + i, 256, 5, 4, n_poly=30, sigma=2.0),
                    256, 5, 4) for i in range(n)]


def burst_pairs(n=32, cache_dir=None):
    """1920x1080 pairs for a burst of concurrent streams, dmax 128, 2 iterations, 16x16 cells."""
    return [_cached(f"burst_{i}", cache_dir,
                    lambda: make_pair("polygon", 1920, 1080, SEED_BASE + 5000 + i, 128, 2, 16, n_poly=20, sigma=2.0),
                    128, 2, 16) for i in range(n)]


# Sizes of the iteration and resolution sweep (the paper's runtime table),
# with the disparity range used at each.
SWEEP_SIZES = [(320, 240, 64), (640, 480, 64), (800, 600, 64), (1280, 720, 128), (1920, 1080, 128)]


def sweep_pairs(W, H, dmax, n=4, cache_dir=None):
    """n polygon-scene pairs of one sweep size (20 planes, noise sigma 2, 16x16
    initial cells); the iteration count is chosen at submit time."""
    return [_cached(f"sweep_{W}x{H}_{i}", cache_dir,
                    lambda: make_pair("polygon", W, H, SEED_BASE + 6000 + 97 * i + W, dmax, 1, 16, n_poly=20, sigma=2.0),
                    dmax, 1, 16) for i in range(n)]


def _cached(key, cache_dir, make, dmax, iters, cell):
    cache_dir = cache_dir or os.environ.get("STEREO_SCENE_CACHE")
    path = os.path.join(cache_dir, f"{key}.npz") if cache_dir else None
    if path and os.path.exists(path):
        z = np.load(path)
        return StereoPair(z["left"], z["right"], z["gt_disp"], z["gt_occ"], dmax, iters, cell)
    p = make()
    if path:
        os.makedirs(cache_dir, exist_ok=True)
        tmp = path + f".{os.getpid()}.npz"
        np.savez(tmp, left=p.left, right=p.right, gt_disp=p.gt_disp, gt_occ=p.gt_occ)
        os.replace(tmp, path)
    return p


def config_pairs(name, n=None, first=0, cache_dir=None):
    """Pairs of one named workload, pair i seeded SEED_BASE + idx*1000 + i.
    With cache_dir (or $STEREO_SCENE_CACHE) rendered pairs are kept as .npz files."""
    cfg = CONFIGS[name]
    count = cfg["n"] if n is None else n
    cache_dir = cache_dir or os.environ.get("STEREO_SCENE_CACHE")
    out = []
    for i in range(first, first + count):
        seed = SEED_BASE + cfg["idx"] * 1000 + i
        path = os.path.join(cache_dir, f"{name}_{seed}.npz") if cache_dir else None
        if path and os.path.exists(path):
            z = np.load(path)
            out.append(StereoPair(z["left"], z["right"], z["gt_disp"], z["gt_occ"], cfg["dmax"], cfg["iters"],
                                  cfg["cell"]))
            continue
        p = make_pair(cfg["kind"], cfg["W"], cfg["H"], seed, cfg["dmax"], cfg["iters"], cfg["cell"], **cfg["kw"])
        if path:
            os.makedirs(cache_dir, exist_ok=True)
            tmp = path + f".{os.getpid()}.npz"
            np.savez(tmp, left=p.left, right=p.right, gt_disp=p.gt_disp, gt_occ=p.gt_occ)
            os.replace(tmp, path)
        out.append(p)
    return out


def integer_shift_pair(W, H, shift, seed=1, dmax=None, texture="noise", flat_left=0):
    """One fronto-parallel plane at an integer disparity, no noise: right(x) = left(x + shift).
    texture="noise" uses the value-noise texture, "iid" independent uniform pixels;
    the first flat_left columns of the scene are black (no corners where the match is out of view)."""
    rng = _rng(seed)
    if texture == "iid":
        img = rng.integers(0, 256, (H, W + shift), dtype=np.uint8)
    else:
        wide = value_noise(*np.meshgrid(np.arange(W + shift, dtype=np.float64) + 777.0,
                                        np.arange(H, dtype=np.float64) + 333.0), int(rng.integers(1, 2**31)))
        img = np.clip(np.rint(wide), 0, 255).astype(np.uint8)
    img[:, :flat_left] = 0
    left = img[:, :W].copy()
    right = img[:, shift:shift + W].copy()  # right(x) = img(x + shift) = left(x + shift)
    # left(u) is seen in the right image at x = u - shift
    gt = np.full((H, W), float(shift), dtype=np.float32)
    occ = np.zeros((H, W), dtype=bool)
    occ[:, :shift] = True
    return StereoPair(left, right, gt, occ, dmax or max(2 * shift, 8), 1, 16)
