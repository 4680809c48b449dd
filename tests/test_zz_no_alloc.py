"""ws_watershed_static: the watershed for callers that cannot allocate device
memory (hosts that pre-reserve the GPU's memory for their own allocator,
latency-critical loops that cannot take cudaMalloc's synchronisation).  Its
scratch is a fixed device array inside the library, shared by every call.

Checked through the C ABI against ws_watershed on two calls in a row, with
tolerance 0 (labels are integer).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2410_08946_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_08946_gb300 import binding
    L = binding.load()
    P = ctypes.c_void_p
    L.ws_watershed_static.argtypes = [P, ctypes.c_int, ctypes.POINTER(binding.ws_shape), ctypes.c_int, P, P, P]
    L.ws_watershed_static.restype = ctypes.c_int
    return L


def _static(lib, grad, conn, stream=None):
    from paper_2410_08946_gb300 import binding
    labels = torch.full(grad.shape, -7, dtype=torch.int32, device="cuda")
    count = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    sh = binding._shape_of(grad.shape)
    s = torch.cuda.current_stream() if stream is None else stream
    st = lib.ws_watershed_static(ctypes.c_void_p(grad.data_ptr()), binding._dtype_code(grad), ctypes.byref(sh),
                                 conn, ctypes.c_void_p(labels.data_ptr()), ctypes.c_void_p(count.data_ptr()),
                                 ctypes.c_void_p(s.cuda_stream))
    return st, labels, count


def test_static_matches_watershed_on_consecutive_calls(lib):
    from paper_2410_08946_gb300 import binding
    cases = [
        (torch.from_numpy(oracle.gradient2d(synth.blob_image(300, 400, 40, seed=5), 4)).cuda(), 8),
        (torch.from_numpy(synth.distance_volume(40, 48, 64, 30, seed=6)).cuda(), 6),
    ]
    with binding.Context(0) as ctx:
        for grad, conn in cases:
            ref_l, ref_k = ctx.watershed(grad, conn)
            ctx.check()
            st, lab, cnt = _static(lib, grad, conn)
            assert st == binding.WS_OK
            torch.cuda.synchronize()
            assert int(cnt.item()) == int(ref_k.item()) > 0
            assert torch.equal(lab, ref_l)


def test_static_repeated_same_input(lib):
    from paper_2410_08946_gb300 import binding
    grad = torch.from_numpy(oracle.gradient2d(synth.blob_image(256, 256, 32, seed=9))).cuda()
    with binding.Context(0) as ctx:
        ref_l, ref_k = ctx.watershed(grad, 4)
        ctx.check()
    for _ in range(2):
        st, lab, cnt = _static(lib, grad, 4)
        assert st == binding.WS_OK
        torch.cuda.synchronize()
        assert int(cnt.item()) == int(ref_k.item())
        assert torch.equal(lab, ref_l)


def test_static_rejects_too_large(lib):
    from paper_2410_08946_gb300 import binding
    grad = torch.zeros((1025, 512), dtype=torch.uint8, device="cuda")   # 524,800 > 524,288 pixels
    st, lab, cnt = _static(lib, grad, 4)
    assert st == binding.WS_ERR_INVALID
    torch.cuda.synchronize()
    assert int(cnt.item()) == -7          # nothing was enqueued
    grad3 = torch.zeros((2, 512, 513), dtype=torch.uint16, device="cuda")
    assert _static(lib, grad3, 6)[0] == binding.WS_ERR_INVALID
