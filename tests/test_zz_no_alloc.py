"""ws_watershed_static: the watershed for callers that cannot allocate device
memory (hosts that pre-reserve the GPU's memory for their own allocator,
latency-critical loops that cannot take cudaMalloc's synchronisation).  Its
scratch is a fixed device array inside the library, shared by every call.

Checked through the C ABI against ws_watershed on two calls in a row and
against the oracle, with tolerance 0 (labels are integer), at the largest
accepted size (including the thinnest 3D shapes, which need the most tiles),
in 2D 4/8 and 3D 6/26 connectivity on uint8 and uint16, with the device's free
memory unchanged across calls.  This file is collected last on purpose."""
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


MAXPX = 524288   # WS_STATIC_MAX_PIXELS


def _check_oracle(lib, arr, conn):
    from paper_2410_08946_gb300 import binding
    grad = torch.from_numpy(np.ascontiguousarray(arr)).cuda()
    st, lab, cnt = _static(lib, grad, conn)
    assert st == binding.WS_OK
    torch.cuda.synchronize()
    ref, K = oracle.watershed(arr, conn)
    assert int(cnt.item()) == K
    assert np.array_equal(lab.cpu().numpy(), ref)


@pytest.mark.parametrize("shape,conn,dtype", [
    ((512, 1024), 4, np.uint8),         # exactly WS_STATIC_MAX_PIXELS
    ((1024, 512), 8, np.uint16),        # 2D uint16
    ((MAXPX, 1, 1), 6, np.uint16),      # one voxel wide and high: the most tiles (32,768)
    ((MAXPX // 2, 2, 1), 26, np.uint8),
    ((1, 1, MAXPX), 6, np.uint8),
    ((64, 64, 128), 26, np.uint16),     # 26-connectivity
])
def test_static_vs_oracle_at_limits(lib, shape, conn, dtype):
    rng = np.random.default_rng(sum(shape) + conn)
    levels = 5 if dtype == np.uint8 else 900
    arr = rng.integers(0, levels, size=shape).astype(dtype)
    _check_oracle(lib, arr, conn)


def test_static_distance_volume_vs_oracle(lib):
    vol = synth.distance_volume(64, 64, 128, 60, seed=14)   # 524,288 voxels
    _check_oracle(lib, vol, 6)


def test_static_allocates_nothing(lib):
    """With no ws_context alive, repeated calls leave the device's free memory
    exactly as it was (the first calls, which load the library's kernels and
    its scratch array, come before the measurement)."""
    from paper_2410_08946_gb300 import binding
    g2 = torch.from_numpy(oracle.gradient2d(synth.blob_image(500, 1000, 60, seed=15))).cuda()
    g3 = torch.from_numpy(synth.distance_volume(32, 64, 200, 20, seed=16)).cuda()
    outs = []
    for grad, conn in ((g2, 4), (g2, 8), (g3, 6), (g3, 26)):
        st, lab, cnt = _static(lib, grad, conn)
        assert st == binding.WS_OK
        outs.append((lab, cnt))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for (grad, conn), (lab, cnt) in zip(((g2, 4), (g2, 8), (g3, 6), (g3, 26)), outs):
            sh = binding._shape_of(grad.shape)
            st = lib.ws_watershed_static(ctypes.c_void_p(grad.data_ptr()), binding._dtype_code(grad),
                                         ctypes.byref(sh), conn, ctypes.c_void_p(lab.data_ptr()),
                                         ctypes.c_void_p(cnt.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert st == binding.WS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
