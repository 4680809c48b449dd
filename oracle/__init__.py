"""CPU oracle for the watershed / waterfall hot path (arXiv 2410.08946).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, sequential, obviously-correct
reference that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It shares no code with the CUDA path and never calls into it.

The arithmetic lives in ``ws_oracle.c`` (plain C, single thread); this module
only compiles it (``build()``), loads it with ctypes and marshals numpy arrays.
Every function cites the passage of the paper it follows in the C source.

Parity status per function (pins are in tests/test_oracle_*.py):
  step1 ............... pinned (Eq. 1 brute force, worked example of Sec. 3.3)
  plateau_distance .... pinned (Sec. 3.3 / Sec. 3.4 worked examples, literal
                        Alg. 1 and Alg. 3 simulations, Floyd-Warshall)
  watershed ........... pinned (exhaustive tiny images vs a literal Alg. 1
                        simulation, invariants, 1D property of Sec. 3.1)
  waterfall ........... pinned (brute force on tiny images, invariants)
  gradient2d .......... pinned by closed forms only (the paper names no operator)
  gradient3d .......... pinned by closed forms, symmetries and the 2D operator
                        on volumes constant along z
  waterfall_reconstruct pinned (hand-derived 1D example, a Python replay of
                        Alg. 5 steps V-VI over all pixel pairs between watersheds)
  region_graph ........ pinned (brute force over all pixel pairs on tiny images,
                        closed-form block grids, a hand-worked example, the
                        lowest-pass rule reproducing the pinned waterfall)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ws_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libws_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ws_oracle.c into libws_oracle.so (portable flags, no intrinsics)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        I = ctypes.c_int
        lib.orc_isqrt_u64.argtypes = [ctypes.c_uint64]
        lib.orc_isqrt_u64.restype = ctypes.c_uint32
        lib.orc_gradient2d.argtypes = [P, i64, i64, I, P]
        lib.orc_step1.argtypes = [P, I, I, P, I, P, P]
        lib.orc_plateau_distance.argtypes = [P, I, I, P, I, P, P]
        lib.orc_watershed.argtypes = [P, I, I, P, I, P, P, P, P, P]
        lib.orc_roots_without_merge.argtypes = [P, I, I, P, I, P]
        lib.orc_waterfall.argtypes = [P, P, I, I, P, I, I, P, P]
        lib.orc_segment.argtypes = [P, I, I, P, I, I, P, P]
        lib.orc_region_graph.argtypes = [P, P, I, I, P, I, P, I, I, i64, P, P, P, i64, P, P, P, P]
        lib.orc_waterfall_reconstruct.argtypes = [P, I, I, P, I, I, P, P]
        lib.orc_gradient3d.argtypes = [P, I, i64, i64, i64, I, P]
        for f in ("orc_gradient2d", "orc_step1", "orc_plateau_distance", "orc_watershed",
                  "orc_roots_without_merge", "orc_waterfall", "orc_segment", "orc_region_graph",
                  "orc_waterfall_reconstruct", "orc_gradient3d"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _geom(grad: np.ndarray):
    """numpy array (H, W) or (D, H, W) -> (ndim, dims[W, H, D] as int64 array)."""
    if grad.ndim == 1:
        grad = grad.reshape(1, -1)
    if grad.ndim == 2:
        H, W = grad.shape
        dims = np.array([W, H, 1], dtype=np.int64)
        return grad, 2, dims
    if grad.ndim == 3:
        D, H, W = grad.shape
        return grad, 3, np.array([W, H, D], dtype=np.int64)
    raise ValueError("image must be 1D, 2D or 3D")


def _prep(grad):
    grad = np.ascontiguousarray(grad)
    if grad.dtype == np.uint8:
        bps = 1
    elif grad.dtype == np.uint16:
        bps = 2
    else:
        raise TypeError("gradient must be uint8 or uint16")
    grad, ndim, dims = _geom(grad)
    return grad, bps, ndim, dims


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"oracle error {rc}")


def isqrt(v: int) -> int:
    return int(_load().orc_isqrt_u64(int(v)))


def gradient2d(img: np.ndarray, quant_shift: int = 0) -> np.ndarray:
    """a0: binomial blur + Sobel + exact isqrt + clip + >> quant_shift."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    if img.ndim == 1:
        img = img.reshape(1, -1)
    H, W = img.shape
    out = np.empty((H, W), dtype=np.uint8)
    _check(_load().orc_gradient2d(_ptr(img), W, H, int(quant_shift), _ptr(out)))
    return out


def gradient3d(vol: np.ndarray, shift: int = 0) -> np.ndarray:
    """3D blur + Sobel + exact isqrt, >> shift, clip 65535: uint16 (D, H, W)."""
    v = np.ascontiguousarray(vol)
    if v.dtype not in (np.uint8, np.uint16) or v.ndim != 3:
        raise TypeError("volume must be a 3D uint8 or uint16 array")
    D, H, W = v.shape
    out = np.empty((D, H, W), dtype=np.uint16)
    _check(_load().orc_gradient3d(_ptr(v), v.dtype.itemsize, W, H, D, int(shift), _ptr(out)))
    return out


def step1(grad: np.ndarray, conn: int):
    """Step I (Eq. 1): returns (S uint8, L int32) with the image's shape."""
    g, bps, ndim, dims = _prep(grad)
    S = np.empty(g.shape, dtype=np.uint8)
    L = np.empty(g.shape, dtype=np.int32)
    _check(_load().orc_step1(_ptr(g), bps, ndim, _ptr(dims), conn, _ptr(S), _ptr(L)))
    return S, L


def plateau_distance(grad: np.ndarray, conn: int, S: np.ndarray | None = None):
    """Step II distances: 0 on state-0 pixels, BFS length on reached plateau
    pixels, -1 elsewhere."""
    g, bps, ndim, dims = _prep(grad)
    if S is None:
        S, _ = step1(g, conn)
    S = np.ascontiguousarray(S, dtype=np.uint8).reshape(g.shape)
    dist = np.empty(g.shape, dtype=np.int32)
    _check(_load().orc_plateau_distance(_ptr(g), bps, ndim, _ptr(dims), conn, _ptr(S), _ptr(dist)))
    return dist


def watershed(grad: np.ndarray, conn: int, debug: bool = False):
    """Steps I-IV + canonical relabel.  Returns (labels int32, K) or, with
    debug=True, (labels, K, S_after_step1, dist, ptr_after_step2)."""
    g, bps, ndim, dims = _prep(grad)
    labels = np.empty(g.shape, dtype=np.int32)
    K = np.zeros(1, dtype=np.int32)
    if debug:
        S = np.empty(g.shape, dtype=np.uint8)
        dist = np.empty(g.shape, dtype=np.int32)
        ptr = np.empty(g.shape, dtype=np.int32)
        _check(_load().orc_watershed(_ptr(g), bps, ndim, _ptr(dims), conn, _ptr(labels), _ptr(K),
                                     _ptr(S), _ptr(dist), _ptr(ptr)))
        return labels, int(K[0]), S, dist, ptr
    _check(_load().orc_watershed(_ptr(g), bps, ndim, _ptr(dims), conn, _ptr(labels), _ptr(K),
                                 None, None, None))
    return labels, int(K[0])


def roots_without_merge(grad: np.ndarray, conn: int) -> np.ndarray:
    """Raw root pixel index after steps I-III (no step IV)."""
    g, bps, ndim, dims = _prep(grad)
    roots = np.empty(g.shape, dtype=np.int32)
    _check(_load().orc_roots_without_merge(_ptr(g), bps, ndim, _ptr(dims), conn, _ptr(roots)))
    return roots


def waterfall(labels0: np.ndarray, grad: np.ndarray, conn: int, NL: int):
    """Graph-form waterfall.  Returns (levels[NL-1, *shape] int32, counts[NL])."""
    g, bps, ndim, dims = _prep(grad)
    L0 = np.ascontiguousarray(labels0, dtype=np.int32).reshape(g.shape)
    levels = np.empty((max(NL - 1, 0),) + g.shape, dtype=np.int32)
    counts = np.empty(NL, dtype=np.int32)
    _check(_load().orc_waterfall(_ptr(L0), _ptr(g), bps, ndim, _ptr(dims), conn, NL,
                                 _ptr(levels), _ptr(counts)))
    return levels, counts


def segment(grad: np.ndarray, conn: int, NL: int):
    """Watershed + waterfall.  Returns (levels[NL, *shape] int32, counts[NL])."""
    g, bps, ndim, dims = _prep(grad)
    levels = np.empty((NL,) + g.shape, dtype=np.int32)
    counts = np.empty(NL, dtype=np.int32)
    _check(_load().orc_segment(_ptr(g), bps, ndim, _ptr(dims), conn, NL, _ptr(levels), _ptr(counts)))
    return levels, counts


def waterfall_reconstruct(grad: np.ndarray, conn: int, NL: int):
    """Paper-literal waterfall (Alg. 4 with Alg. 5's image reconstruction).
    Returns (levels[NL, *shape] int32, counts[NL])."""
    g, bps, ndim, dims = _prep(grad)
    levels = np.empty((NL,) + g.shape, dtype=np.int32)
    counts = np.empty(NL, dtype=np.int32)
    _check(_load().orc_waterfall_reconstruct(_ptr(g), bps, ndim, _ptr(dims), conn, NL, _ptr(levels),
                                             _ptr(counts)))
    return levels, counts


def region_graph(labels: np.ndarray, grad: np.ndarray, conn: int, values: np.ndarray | None = None):
    """Region graph of one labelling (Sec. 6 node/edge export, Alg. 5 step V
    pass values).  labels: ids >= 0 with the gradient's shape; values: None or
    (C, *shape) uint8/uint16 (a single plane may omit C).  Returns a dict with
    row_ptr int64[K+1], col int32[nnz], pass uint32[nnz] (symmetric CSR, columns
    ascending), size int64[K], sum uint64[K, C], mean float64[K, C]; K = max id + 1."""
    g, bps, ndim, dims = _prep(grad)
    L = np.ascontiguousarray(labels, dtype=np.int32).reshape(g.shape)
    N = L.size
    if L.min() < 0:
        raise ValueError("labels must be >= 0")
    K = int(L.max()) + 1
    if values is None:
        C, vbps, v = 0, 1, np.zeros(1, dtype=np.uint8)
    else:
        v = np.ascontiguousarray(values)
        if v.dtype not in (np.uint8, np.uint16):
            raise TypeError("values must be uint8 or uint16")
        v = v.reshape(-1, N)
        C, vbps = v.shape[0], v.dtype.itemsize
    if conn not in (4, 8, 6, 26):
        raise ValueError("connectivity must be 4, 8, 6 or 26")
    cap = N * conn  # one record per ordered neighbour pair at most
    row_ptr = np.empty(K + 1, dtype=np.int64)
    col = np.empty(max(cap, 1), dtype=np.int32)
    pas = np.empty(max(cap, 1), dtype=np.uint32)
    nnz = np.zeros(1, dtype=np.int64)
    size = np.empty(K, dtype=np.int64)
    ssum = np.empty((K, max(C, 1)), dtype=np.uint64)
    mean = np.empty((K, max(C, 1)), dtype=np.float64)
    _check(_load().orc_region_graph(_ptr(L), _ptr(g), bps, ndim, _ptr(dims), conn, _ptr(v), vbps, C, K,
                                    _ptr(row_ptr), _ptr(col), _ptr(pas), cap, _ptr(nnz), _ptr(size),
                                    _ptr(ssum), _ptr(mean)))
    n = int(nnz[0])
    return {"row_ptr": row_ptr, "col": col[:n].copy(), "pass": pas[:n].copy(), "size": size,
            "sum": ssum[:, :C].copy(), "mean": mean[:, :C].copy()}
