"""Thin ctypes binding of libws (the C ABI in include/ws.h).

Argument marshalling only: every step of the watershed / waterfall runs in the
library's CUDA kernels.  Device buffers are torch CUDA tensors (passed by
``data_ptr()``), the stream is torch's current stream unless given.  There is
no CPU fallback: if libws.so is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libws.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ws.h")

WS_OK, WS_ERR_INVALID, WS_ERR_UNSUPPORTED, WS_ERR_OOM, WS_ERR_CUDA = 0, 1, 2, 3, 4
WS_ERR_NONCONVERGED, WS_ERR_TIMEOUT, WS_ERR_NOT_READY, WS_ERR_CANCELLED = 5, 6, 7, 8
WS_U8, WS_U16 = 0, 1
STATUS_NAMES = {0: "WS_OK", 1: "WS_ERR_INVALID", 2: "WS_ERR_UNSUPPORTED", 3: "WS_ERR_OOM", 4: "WS_ERR_CUDA",
                5: "WS_ERR_NONCONVERGED", 6: "WS_ERR_TIMEOUT", 7: "WS_ERR_NOT_READY", 8: "WS_ERR_CANCELLED"}


class WsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ws_shape(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("pad_", ctypes.c_int32), ("dims", ctypes.c_int64 * 3)]


class ws_item(ctypes.Structure):
    _fields_ = [("grad_d", ctypes.c_void_p), ("shape", ws_shape), ("levels_d", ctypes.c_void_p),
                ("counts_d", ctypes.c_void_p)]


class ws_request(ctypes.Structure):
    _fields_ = [("grad", ctypes.c_void_p), ("on_host", ctypes.c_int32), ("connectivity", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("NL", ctypes.c_int32), ("shape", ws_shape),
                ("levels", ctypes.c_void_p), ("counts", ctypes.c_void_p)]


class ws_tuning(ctypes.Structure):
    _fields_ = [("plateau_round_cap", ctypes.c_int32), ("jump_round_cap", ctypes.c_int32),
                ("jumps_per_round", ctypes.c_int32), ("barrier_timeout_ms", ctypes.c_int32),
                ("edge_capacity", ctypes.c_int64), ("levels_ctas_per_sm", ctypes.c_int32),
                ("barrier_withhold", ctypes.c_int32), ("tile_shape", ctypes.c_int32), ("pad_", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def declared_symbols(header: str = HEADER):
    """Names of the functions include/ws.h declares."""
    txt = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:ws_status|void|const char \*|size_t|int|unsigned long long)\s*\*?\s*(ws_\w+)\s*\(",
                                 txt, flags=re.M)))


def load(path: str = LIB_PATH):
    """Loads libws.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libws.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        SH = ctypes.POINTER(ws_shape)
        sig = {
            "ws_context_create": ([ctypes.POINTER(P), I, S], I),
            "ws_context_destroy": ([P], None),
            "ws_context_check": ([P, P], I),
            "ws_last_error": ([P], ctypes.c_char_p),
            "ws_context_set_tuning": ([P, ctypes.POINTER(ws_tuning)], I),
            "ws_context_workspace_bytes": ([P], S),
            "ws_gradient": ([P, P, SH, I, P, P], I),
            "ws_watershed": ([P, P, I, SH, I, P, P, P], I),
            "ws_waterfall": ([P, P, P, I, SH, I, I, P, P, P], I),
            "ws_segment": ([P, P, I, SH, I, I, P, P, P], I),
            "ws_segment_host": ([P, P, I, SH, I, I, P, P, P], I),
            "ws_step1": ([P, P, I, SH, I, P, P, P], I),
            "ws_plateau_distance": ([P, P, I, SH, I, P, P], I),
            "ws_context_set_profiling": ([P, I], I),
            "ws_phase_count": ([], I),
            "ws_phase_name": ([I], ctypes.c_char_p),
            "ws_context_phase_times": ([P, P, P, I], I),
            "ws_context_launches": ([P], ctypes.c_ulonglong),
            "ws_context_counters": ([P, P, P, I], I),
            "ws_segment_batch": ([P, I, ctypes.POINTER(ws_item), I, I, I, P], I),
            "ws_graph_create": ([P, I, ctypes.POINTER(ws_item), I, I, I, P, ctypes.POINTER(P)], I),
            "ws_graph_launch": ([P, P], I),
            "ws_graph_destroy": ([P], None),
            "ws_server_create": ([ctypes.POINTER(P), I, S, I, I], I),
            "ws_submit": ([P, ctypes.POINTER(ws_request), ctypes.POINTER(ctypes.c_uint64)], I),
            "ws_poll": ([P, ctypes.c_uint64, ctypes.c_int64], I),
            "ws_cancel": ([P, ctypes.c_uint64], I),
            "ws_server_destroy": ([P], None),
            "ws_region_graph": ([P, P, P, I, SH, I, P, I, I, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int64), P], I),
            "ws_region_graph_read": ([P, P, P, P, P, P, P, P], I),
            "ws_waterfall_reconstruct": ([P, P, I, SH, I, I, P, P, P], I),
            "ws_gradient3d": ([P, P, I, SH, I, P, P], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _shape_of(shape) -> ws_shape:
    shape = tuple(int(s) for s in shape)
    s = ws_shape()
    if len(shape) == 1:
        shape = (1,) + shape
    if len(shape) == 2:
        s.ndim = 2
        s.dims[0], s.dims[1], s.dims[2] = shape[1], shape[0], 1
    elif len(shape) == 3:
        s.ndim = 3
        s.dims[0], s.dims[1], s.dims[2] = shape[2], shape[1], shape[0]
    else:
        raise ValueError("images are 2D (H, W) or 3D (D, H, W)")
    return s


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.uint8:
        return WS_U8
    if t.dtype == torch.uint16:
        return WS_U16
    raise TypeError("gradient must be uint8 or uint16")


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """A libws context (workspace + device status word) on one GPU."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        self.lib = load()
        self.handle = ctypes.c_void_p()
        st = self.lib.ws_context_create(ctypes.byref(self.handle), int(device), int(budget_bytes))
        if st != WS_OK:
            raise WsError(st, "ws_context_create failed")
        self.device = device

    def close(self):
        if self.handle:
            self.lib.ws_context_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- plumbing ---------------------------------------------------------
    def last_error(self) -> str:
        return (self.lib.ws_last_error(self.handle) or b"").decode()

    def _ok(self, st: int):
        if st != WS_OK:
            raise WsError(st, self.last_error())

    def check(self, stream=None):
        """Synchronise the stream and raise if the device recorded an error."""
        self._ok(self.lib.ws_context_check(self.handle, _stream(stream)))

    def set_tuning(self, **kw):
        t = ws_tuning(**kw)
        self._ok(self.lib.ws_context_set_tuning(self.handle, ctypes.byref(t)))

    def workspace_bytes(self) -> int:
        return int(self.lib.ws_context_workspace_bytes(self.handle))

    def set_profiling(self, on: bool = True):
        self._ok(self.lib.ws_context_set_profiling(self.handle, 1 if on else 0))

    def phase_times(self):
        """{phase name: (total ms, instances)} since the last call (waits for the events)."""
        n = int(self.lib.ws_phase_count())
        ms = (ctypes.c_double * n)()
        calls = (ctypes.c_longlong * n)()
        self._ok(self.lib.ws_context_phase_times(self.handle, ms, calls, n))
        return {self.lib.ws_phase_name(i).decode(): (ms[i], calls[i]) for i in range(n)}

    def launches(self) -> int:
        """Kernels this context has enqueued so far."""
        return int(self.lib.ws_context_launches(self.handle))

    COUNTERS = ("plateau_rounds", "jump_rounds", "edge_records", "basins", "path_ends", "plateau_tiles",
                "plateau_pixels")

    def counters(self, stream=None) -> dict:
        """The device's counts for the last watershed call (waits for the stream)."""
        out = (ctypes.c_int64 * len(self.COUNTERS))()
        self._ok(self.lib.ws_context_counters(self.handle, _stream(stream), out, len(self.COUNTERS)))
        return dict(zip(self.COUNTERS, (int(v) for v in out)))

    # -- entry points -------------------------------------------------------
    def gradient(self, img, quant_shift: int = 0, out=None, stream=None):
        import torch
        if img.dtype != torch.uint8 or img.dim() != 2:
            raise TypeError("gradient takes a 2D uint8 image")
        out = torch.empty_like(img) if out is None else out
        sh = _shape_of(img.shape)
        self._ok(self.lib.ws_gradient(self.handle, _dev(img), ctypes.byref(sh), int(quant_shift), _dev(out),
                                      _stream(stream)))
        return out

    def gradient3d(self, vol, shift: int = 0, out=None, stream=None):
        """3D blur + Sobel magnitude of a uint8 / uint16 volume -> uint16 volume."""
        import torch
        if vol.dim() != 3:
            raise TypeError("gradient3d takes a 3D volume")
        out = torch.empty(vol.shape, dtype=torch.uint16, device=vol.device) if out is None else out
        sh = _shape_of(vol.shape)
        self._ok(self.lib.ws_gradient3d(self.handle, _dev(vol), _dtype_code(vol), ctypes.byref(sh), int(shift),
                                        _dev(out), _stream(stream)))
        return out

    def step1(self, grad, conn: int, stream=None):
        import torch
        states = torch.empty(grad.shape, dtype=torch.uint8, device=grad.device)
        arrows = torch.empty(grad.shape, dtype=torch.int32, device=grad.device)
        sh = _shape_of(grad.shape)
        self._ok(self.lib.ws_step1(self.handle, _dev(grad), _dtype_code(grad), ctypes.byref(sh), int(conn),
                                   _dev(states), _dev(arrows), _stream(stream)))
        return states, arrows

    def plateau_distance(self, grad, conn: int, stream=None):
        import torch
        dist = torch.empty(grad.shape, dtype=torch.int32, device=grad.device)
        sh = _shape_of(grad.shape)
        self._ok(self.lib.ws_plateau_distance(self.handle, _dev(grad), _dtype_code(grad), ctypes.byref(sh),
                                              int(conn), _dev(dist), _stream(stream)))
        return dist

    def watershed(self, grad, conn: int, labels=None, count=None, stream=None):
        import torch
        labels = torch.empty(grad.shape, dtype=torch.int32, device=grad.device) if labels is None else labels
        count = torch.empty(1, dtype=torch.int32, device=grad.device) if count is None else count
        sh = _shape_of(grad.shape)
        self._ok(self.lib.ws_watershed(self.handle, _dev(grad), _dtype_code(grad), ctypes.byref(sh), int(conn),
                                       _dev(labels), _dev(count), _stream(stream)))
        return labels, count

    def waterfall(self, labels0, grad, conn: int, NL: int, levels=None, counts=None, stream=None):
        import torch
        if levels is None:
            levels = torch.empty((max(NL - 1, 1),) + tuple(grad.shape), dtype=torch.int32, device=grad.device)
        counts = torch.empty(NL, dtype=torch.int32, device=grad.device) if counts is None else counts
        sh = _shape_of(grad.shape)
        self._ok(self.lib.ws_waterfall(self.handle, _dev(labels0), _dev(grad), _dtype_code(grad), ctypes.byref(sh),
                                       int(conn), int(NL), _dev(levels), _dev(counts), _stream(stream)))
        return levels[: NL - 1], counts

    def waterfall_reconstruct(self, grad, conn: int, NL: int, levels=None, counts=None, stream=None):
        """Paper-literal waterfall (ws_waterfall_reconstruct): NL label planes."""
        import torch
        if levels is None:
            levels = torch.empty((NL,) + tuple(grad.shape), dtype=torch.int32, device=grad.device)
        counts = torch.empty(NL, dtype=torch.int32, device=grad.device) if counts is None else counts
        sh = _shape_of(grad.shape)
        self._ok(self.lib.ws_waterfall_reconstruct(self.handle, _dev(grad), _dtype_code(grad), ctypes.byref(sh),
                                                   int(conn), int(NL), _dev(levels), _dev(counts), _stream(stream)))
        return levels, counts

    def region_graph(self, labels, grad, conn: int, values=None, stream=None):
        """Region graph of one labelling (ws_region_graph + ws_region_graph_read).
        values: None or a (C, *shape) / shape-sized uint8 or uint16 CUDA tensor.
        Returns a dict of CUDA tensors: row_ptr int64[K+1], col int32[nnz],
        pass int32[nnz] (the uint32 pass values, all below 2^16), size int64[K],
        sum int64[K, C] (uint64 sums, all below 2^63), mean float64[K, C]."""
        import torch
        if labels.dtype != torch.int32 or tuple(labels.shape) != tuple(grad.shape):
            raise TypeError("labels must be int32 with the gradient's shape")
        C, vptr, vcode = 0, None, WS_U8
        if values is not None:
            if values.dtype not in (torch.uint8, torch.uint16):
                raise TypeError("values must be uint8 or uint16")
            C = values.numel() // grad.numel()
            if C * grad.numel() != values.numel():
                raise ValueError("values must hold whole planes of the image")
            vptr, vcode = _dev(values), _dtype_code(values)
        sh = _shape_of(grad.shape)
        K, nnz = ctypes.c_int64(), ctypes.c_int64()
        st = _stream(stream)
        self._ok(self.lib.ws_region_graph(self.handle, _dev(labels), _dev(grad), _dtype_code(grad),
                                          ctypes.byref(sh), int(conn), vptr, vcode, C, ctypes.byref(K),
                                          ctypes.byref(nnz), st))
        K, nnz = K.value, nnz.value
        dev = grad.device
        out = {"row_ptr": torch.empty(K + 1, dtype=torch.int64, device=dev),
               "col": torch.empty(max(nnz, 1), dtype=torch.int32, device=dev),
               "pass": torch.empty(max(nnz, 1), dtype=torch.int32, device=dev),
               "size": torch.empty(K, dtype=torch.int64, device=dev),
               "sum": torch.empty((K, max(C, 1)), dtype=torch.int64, device=dev),
               "mean": torch.empty((K, max(C, 1)), dtype=torch.float64, device=dev)}
        self._ok(self.lib.ws_region_graph_read(self.handle, _dev(out["row_ptr"]), _dev(out["col"]),
                                               _dev(out["pass"]), _dev(out["size"]),
                                               _dev(out["sum"]) if C else None,
                                               _dev(out["mean"]) if C else None, st))
        out["col"], out["pass"] = out["col"][:nnz], out["pass"][:nnz]
        out["sum"], out["mean"] = out["sum"][:, :C], out["mean"][:, :C]
        return out

    def segment(self, grad, conn: int, NL: int, levels=None, counts=None, stream=None):
        import torch
        if levels is None:
            levels = torch.empty((NL,) + tuple(grad.shape), dtype=torch.int32, device=grad.device)
        counts = torch.empty(NL, dtype=torch.int32, device=grad.device) if counts is None else counts
        sh = _shape_of(grad.shape)
        self._ok(self.lib.ws_segment(self.handle, _dev(grad), _dtype_code(grad), ctypes.byref(sh), int(conn),
                                     int(NL), _dev(levels), _dev(counts), _stream(stream)))
        return levels, counts

    def _items(self, grads, NL, levels=None, counts=None):
        import torch
        n = len(grads)
        if levels is None:
            levels = [torch.empty((NL,) + tuple(g.shape), dtype=torch.int32, device=g.device) for g in grads]
        if counts is None:
            counts = [torch.empty(NL, dtype=torch.int32, device=g.device) for g in grads]
        arr = (ws_item * n)()
        for i, g in enumerate(grads):
            arr[i].grad_d = _dev(g)
            arr[i].shape = _shape_of(g.shape)
            arr[i].levels_d = _dev(levels[i])
            arr[i].counts_d = _dev(counts[i])
        dt = _dtype_code(grads[0])
        if any(_dtype_code(g) != dt for g in grads):
            raise TypeError("every image of a batch must have the same dtype")
        return arr, dt, levels, counts

    def segment_batch(self, grads, conn: int, NL: int, levels=None, counts=None, stream=None):
        """ws_segment for a list of images at once; returns (levels list, counts list)."""
        arr, dt, levels, counts = self._items(grads, NL, levels, counts)
        self._ok(self.lib.ws_segment_batch(self.handle, len(grads), arr, dt, int(conn), int(NL), _stream(stream)))
        return levels, counts

    def graph(self, grads, conn: int, NL: int, levels=None, counts=None, stream=None):
        """Records the batch into a CUDA graph; returns a BatchGraph (with .levels, .counts)."""
        arr, dt, levels, counts = self._items(grads, NL, levels, counts)
        h = ctypes.c_void_p()
        self._ok(self.lib.ws_graph_create(self.handle, len(grads), arr, dt, int(conn), int(NL), _stream(stream),
                                          ctypes.byref(h)))
        return BatchGraph(self, h, levels, counts)

    def segment_host(self, grad_h, conn: int, NL: int, levels_h=None, counts_h=None, stream=None):
        """grad_h, levels_h, counts_h: CPU tensors (pinned for speed).  Blocks until done."""
        import torch
        if grad_h.is_cuda or not grad_h.is_contiguous():
            raise ValueError("segment_host takes a contiguous CPU tensor")
        if levels_h is None:
            levels_h = torch.empty((NL,) + tuple(grad_h.shape), dtype=torch.int32, pin_memory=True)
        if counts_h is None:
            counts_h = torch.empty(NL, dtype=torch.int32)
        sh = _shape_of(grad_h.shape)
        self._ok(self.lib.ws_segment_host(self.handle, ctypes.c_void_p(grad_h.data_ptr()), _dtype_code(grad_h),
                                          ctypes.byref(sh), int(conn), int(NL), ctypes.c_void_p(levels_h.data_ptr()),
                                          ctypes.c_void_p(counts_h.data_ptr()), _stream(stream)))
        return levels_h, counts_h


class BatchGraph:
    """A batch recorded as a CUDA graph (ws_graph_create); launch() replays it."""

    def __init__(self, ctx, handle, levels, counts):
        self.ctx, self.handle, self.levels, self.counts = ctx, handle, levels, counts

    def launch(self, stream=None):
        self.ctx._ok(self.ctx.lib.ws_graph_launch(self.handle, _stream(stream)))

    def close(self):
        if self.handle:
            self.ctx.lib.ws_graph_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A libws request loop (ws_server_*): continuous batching over lanes."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, lanes: int = 4, max_batch: int = 64):
        self.lib = load()
        self.handle = ctypes.c_void_p()
        st = self.lib.ws_server_create(ctypes.byref(self.handle), int(device), int(budget_bytes), int(lanes),
                                       int(max_batch))
        if st != WS_OK:
            raise WsError(st, "ws_server_create failed")
        self._keep = {}

    def submit(self, grad, conn: int, NL: int, levels=None, counts=None) -> int:
        """Queues one image (CPU tensor: host request, CUDA tensor: device request).
        Returns the ticket; outputs are kept alive until the ticket is polled."""
        import torch
        on_host = not grad.is_cuda
        if levels is None:
            levels = torch.empty((NL,) + tuple(grad.shape), dtype=torch.int32, device=grad.device,
                                 pin_memory=on_host)
        if counts is None:
            counts = torch.empty(NL, dtype=torch.int32, device=grad.device, pin_memory=on_host)
        r = ws_request()
        r.grad = ctypes.c_void_p(grad.data_ptr())
        r.on_host = 1 if on_host else 0
        r.connectivity = int(conn)
        r.dtype = _dtype_code(grad)
        r.NL = int(NL)
        r.shape = _shape_of(grad.shape)
        r.levels = ctypes.c_void_p(levels.data_ptr())
        r.counts = ctypes.c_void_p(counts.data_ptr())
        t = ctypes.c_uint64()
        st = self.lib.ws_submit(self.handle, ctypes.byref(r), ctypes.byref(t))
        if st != WS_OK:
            raise WsError(st, "ws_submit failed")
        self._keep[t.value] = (grad, levels, counts)
        return t.value

    def poll(self, ticket: int, timeout_us: int = -1):
        """Returns (status, levels, counts); outputs are meaningful when status == WS_OK."""
        st = self.lib.ws_poll(self.handle, ctypes.c_uint64(ticket), int(timeout_us))
        if st == WS_ERR_NOT_READY:
            return st, None, None
        _, levels, counts = self._keep.pop(ticket, (None, None, None))
        return st, levels, counts

    def cancel(self, ticket: int) -> int:
        return self.lib.ws_cancel(self.handle, ctypes.c_uint64(ticket))

    def close(self):
        if self.handle:
            self.lib.ws_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
