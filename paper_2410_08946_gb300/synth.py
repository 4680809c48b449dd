"""Seeded synthetic inputs for the watershed / waterfall workloads.

This module generates *inputs only*; it holds none of the method's arithmetic
(no gradient operator, no watershed step).  Both the CUDA path and the CPU
oracle consume exactly the arrays produced here.

All randomness comes from one counter-based generator, SplitMix64 (Steele,
Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
value i of stream s under seed k is splitmix64(key(k, s) + i).  It is fully
defined here, so the inputs do not depend on numpy's RNG versions.

Workloads (sizes and value distributions follow the paper's test images:
2D 256^2..4000^2 greyscale, 3D up to 8e8 voxels; the datasets themselves are
not available, so these seeded stand-ins are used):

  blob_image          sum of Gaussian blobs (sigma U[4,20] px, amplitude
                      U[40,200]) + uniform integer noise U{0..16}, uint8
  distance_volume     distance to the nearest of n random seed points, scaled
                      to [0, 65535], + uniform integer noise U{0..64}, uint16
  batch_shapes        side lengths log-uniform in [lo, hi]
  request_stream      Poisson arrivals with a 2D / 3D mix
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

BASE_SEED = 2410089460
_M64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser of x + golden gamma, vectorised over uint64."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> int:
    k = splitmix64(np.uint64((seed * 0x9E3779B1 + stream * 0x85EBCA77) & _M64))
    return int(k)


def raw(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    k = _key(seed, stream)
    idx = np.arange(start, start + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64(idx + np.uint64(k))


def uniform(seed: int, stream: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    u = (raw(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return lo + (hi - lo) * u


def integers(seed: int, stream: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Uniform integers in [lo, hi] (inclusive), by modulo reduction."""
    span = np.uint64(hi - lo + 1)
    return (raw(seed, stream, n) % span).astype(np.int64) + lo


# --------------------------------------------------------------------------
# 2D: Gaussian blobs + noise (uint8 greyscale image)
# --------------------------------------------------------------------------

def blob_image(H: int, W: int, n_blobs: int, seed: int, noise_max: int = 16,
               sigma=(4.0, 20.0), amp=(40.0, 200.0)) -> np.ndarray:
    """uint8 image = clip(rint(sum_b A_b exp(-r^2 / (2 sigma_b^2))) + U{0..noise_max}, 0, 255).

    Each blob is evaluated on the window |dx|, |dy| <= ceil(5 sigma) around its
    centre (the tail beyond contributes < 7.5e-4 grey levels); float64."""
    cx = uniform(seed, 1, n_blobs, 0.0, float(W))
    cy = uniform(seed, 2, n_blobs, 0.0, float(H))
    sg = uniform(seed, 3, n_blobs, sigma[0], sigma[1])
    am = uniform(seed, 4, n_blobs, amp[0], amp[1])
    acc = np.zeros((H, W), dtype=np.float64)
    for b in range(n_blobs):
        r = int(math.ceil(5.0 * sg[b]))
        x0, x1 = max(0, int(math.floor(cx[b])) - r), min(W, int(math.floor(cx[b])) + r + 1)
        y0, y1 = max(0, int(math.floor(cy[b])) - r), min(H, int(math.floor(cy[b])) + r + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        xs = np.arange(x0, x1, dtype=np.float64) - cx[b]
        ys = np.arange(y0, y1, dtype=np.float64) - cy[b]
        inv = 1.0 / (2.0 * sg[b] * sg[b])
        acc[y0:y1, x0:x1] += am[b] * np.exp(-(ys[:, None] ** 2) * inv) * np.exp(-(xs[None, :] ** 2) * inv)
    noise = integers(seed, 5, H * W, 0, noise_max).reshape(H, W)
    return np.clip(np.rint(acc) + noise, 0, 255).astype(np.uint8)


def blob_count_for(H: int, W: int) -> int:
    """Blob count for an image of H x W: 32 per 256^2, clamped to [8, 2000]."""
    return int(min(2000, max(8, round(32 * W * H / 65536))))


# --------------------------------------------------------------------------
# 3D: distance to random seed points + noise (uint16 volume)
# --------------------------------------------------------------------------

_HERE = os.path.dirname(os.path.abspath(__file__))
_SYN_SRC = os.path.join(_HERE, "csrc", "synth_edt.c")
_SYN_LIB = os.path.join(_HERE, "libwssynth.so")
_syn = None
_syn_lock = threading.Lock()


def build_synth(force: bool = False) -> str:
    if (not force and os.path.exists(_SYN_LIB)
            and os.path.getmtime(_SYN_LIB) >= os.path.getmtime(_SYN_SRC)):
        return _SYN_LIB
    tmp = _SYN_LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp,
                           _SYN_SRC, "-lm"])
    os.replace(tmp, _SYN_LIB)
    return _SYN_LIB


def _synlib():
    global _syn
    with _syn_lock:
        if _syn is None:
            build_synth()
            lib = ctypes.CDLL(_SYN_LIB)
            P, i64 = ctypes.c_void_p, ctypes.c_int64
            lib.synth_edt3d.argtypes = [i64, i64, i64, P, i64, P, ctypes.c_int]
            lib.synth_distance_volume.argtypes = [i64, i64, i64, P, i64, ctypes.c_uint64,
                                                  ctypes.c_int, P, ctypes.c_int]
            lib.synth_edt3d.restype = ctypes.c_int
            lib.synth_distance_volume.restype = ctypes.c_int
            _syn = lib
        return _syn


def seed_points(D: int, H: int, W: int, n: int, seed: int) -> np.ndarray:
    """n seed points at uniform integer coordinates, int64 array (n, 3) of (x, y, z)."""
    xs = integers(seed, 11, n, 0, W - 1)
    ys = integers(seed, 12, n, 0, H - 1)
    zs = integers(seed, 13, n, 0, D - 1)
    return np.ascontiguousarray(np.stack([xs, ys, zs], axis=1).astype(np.int64))


def squared_edt(D: int, H: int, W: int, seeds: np.ndarray, threads: int | None = None) -> np.ndarray:
    out = np.empty((D, H, W), dtype=np.uint32)
    s = np.ascontiguousarray(seeds, dtype=np.int64)
    rc = _synlib().synth_edt3d(W, H, D, s.ctypes.data, len(s), out.ctypes.data,
                               threads or min(32, os.cpu_count() or 1))
    if rc != 0:
        raise RuntimeError(f"synth_edt3d failed ({rc})")
    return out


def distance_volume(D: int, H: int, W: int, n_seeds: int, seed: int, noise_levels: int = 65,
                    threads: int | None = None) -> np.ndarray:
    """uint16 volume: isqrt(d^2 * 65535^2 / max d^2) + U{0..noise_levels-1}, saturated."""
    seeds = seed_points(D, H, W, n_seeds, seed)
    out = np.empty((D, H, W), dtype=np.uint16)
    key = _key(seed, 14)
    rc = _synlib().synth_distance_volume(W, H, D, seeds.ctypes.data, len(seeds), key, noise_levels,
                                         out.ctypes.data, threads or min(32, os.cpu_count() or 1))
    if rc != 0:
        raise RuntimeError(f"synth_distance_volume failed ({rc})")
    return out


def distance_volume_reference(D: int, H: int, W: int, n_seeds: int, seed: int,
                              noise_levels: int = 65) -> np.ndarray:
    """Brute-force numpy restatement of distance_volume (small sizes only)."""
    seeds = seed_points(D, H, W, n_seeds, seed)
    z, y, x = np.meshgrid(np.arange(D), np.arange(H), np.arange(W), indexing="ij")
    d2 = np.full((D, H, W), np.iinfo(np.int64).max, dtype=np.int64)
    for sx, sy, sz in seeds.tolist():
        d2 = np.minimum(d2, (x - sx) ** 2 + (y - sy) ** 2 + (z - sz) ** 2)
    d2max = max(int(d2.max()), 1)
    flat = d2.ravel()
    base = np.array([math.isqrt(int(v) * 65535 * 65535 // d2max) for v in flat.tolist()], dtype=np.int64)
    key = _key(seed, 14)
    idx = np.arange(flat.size, dtype=np.uint64)
    with np.errstate(over="ignore"):
        nz = (splitmix64(idx + np.uint64(key)) % np.uint64(noise_levels)).astype(np.int64)
    return np.minimum(base + nz, 65535).astype(np.uint16).reshape(D, H, W)


# --------------------------------------------------------------------------
# batches and request streams
# --------------------------------------------------------------------------

def log_uniform_sides(n: int, lo: int, hi: int, seed: int, stream: int) -> np.ndarray:
    u = uniform(seed, stream, n)
    return np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def batch_shapes(n: int, lo: int, hi: int, seed: int):
    """n (H, W) pairs, each side independently log-uniform in [lo, hi]."""
    hs = log_uniform_sides(n, lo, hi, seed, 21)
    ws = log_uniform_sides(n, lo, hi, seed, 22)
    return [(int(h), int(w)) for h, w in zip(hs, ws)]


def request_stream(rate_hz: float, duration_s: float, seed: int, frac_3d: float = 0.2,
                   side2d=(256, 4096), side3d=(64, 256)):
    """Poisson arrivals: list of dicts {t, kind, shape}.  Exponential gaps,
    a Bernoulli(frac_3d) 2D/3D mix, sides independently log-uniform."""
    n_max = int(rate_hz * duration_s * 2 + 64)
    gaps = -np.log1p(-uniform(seed, 31, n_max)) / rate_hz
    t = np.cumsum(gaps)
    n = int(np.searchsorted(t, duration_s))
    kind = uniform(seed, 32, n) < frac_3d
    out = []
    s2 = [log_uniform_sides(n, side2d[0], side2d[1], seed, 33 + i) for i in range(2)]
    s3 = [log_uniform_sides(n, side3d[0], side3d[1], seed, 35 + i) for i in range(3)]
    for i in range(n):
        if kind[i]:
            out.append(dict(t=float(t[i]), kind="3d", shape=(int(s3[2][i]), int(s3[1][i]), int(s3[0][i])),
                            seed=seed * 100003 + i))
        else:
            out.append(dict(t=float(t[i]), kind="2d", shape=(int(s2[1][i]), int(s2[0][i])),
                            seed=seed * 100003 + i))
    return out


# --------------------------------------------------------------------------
# the batch (config 3) and the request stream (config 4): crops of one large
# 2D blob image and of one 3D distance volume
# --------------------------------------------------------------------------

CROP_SIDE = 4096                   # the 2D image the batch and the requests are cut from
CROP_BLOBS = 8192                  # 32 blobs per 256^2, the small-image density
BATCH_POOL_SEED = BASE_SEED + 3    # the batch's 4096^2 image
BATCH_SHAPE_SEED = BASE_SEED + 5   # the batch's crop sides and offsets
SERVE_SEED = BASE_SEED + 6         # the request stream, its 2D image and its 3D volume
SERVE_VOLUME_SIDE = 256
SERVE_VOLUME_SEEDS = 1050          # 50,000 seeds scaled by volume from 928^3 to 256^3


def crop_pool_image(seed: int) -> np.ndarray:
    """The CROP_SIDE^2 uint8 blob image that 2D batch images and requests are
    cut from (its gradient, rather: callers crop the gradient)."""
    return blob_image(CROP_SIDE, CROP_SIDE, CROP_BLOBS, seed)


def batch_windows(n: int, seed: int = BATCH_SHAPE_SEED, lo: int = 64, hi: int = 2048):
    """n crop windows (y, x, h, w) of the CROP_SIDE^2 image: sides
    independently log-uniform in [lo, hi], offsets uniform in [0, CROP_SIDE - hi]."""
    shapes = batch_shapes(n, lo, hi, seed)
    offs = integers(seed, 41, 2 * n, 0, CROP_SIDE - hi)
    return [(int(offs[2 * i]), int(offs[2 * i + 1]), h, w) for i, (h, w) in enumerate(shapes)]


def request_window_2d(i: int, h: int, w: int):
    """Crop origin (y, x) of 2D request i (h x w) in the CROP_SIDE^2 image."""
    return (i * 7919) % (CROP_SIDE + 1 - h), (i * 104729) % (CROP_SIDE + 1 - w)
