"""26-connectivity in 3D (every voxel of the 3x3x3 cube is a neighbour):
watershed and watershed + waterfall against the oracle, tolerance 0, on
random volumes spanning several tiles with ragged tails, distance volumes on
both staging paths (TMA needs rows of 16-byte multiples), uint8 volumes with
plateaux, batches, and the allocation-free entry point."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2410_08946_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_08946_gb300 import binding
    c = binding.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("shape,levels", [((1, 1, 1), 3), ((2, 3, 4), 3), ((9, 20, 18), 2), ((17, 19, 40), 4),
                                          ((33, 34, 35), 3), ((10, 10, 10), 65536)])
def test_watershed_26_random(ctx, shape, levels):
    rng = np.random.default_rng(hash((shape, levels, 26)) % 2**32)
    v = rng.integers(0, levels, size=shape).astype(np.uint16)
    L, K = oracle.watershed(v, 26)
    l_d, k_d = ctx.watershed(dev(v), 26)
    ctx.check()
    assert int(k_d.cpu()[0]) == K
    assert np.array_equal(l_d.cpu().numpy(), L)


@pytest.mark.parametrize("W", [64, 60])
@pytest.mark.parametrize("seeds", [12, 400])
def test_segment_26_distance(ctx, W, seeds):
    v = synth.distance_volume(30, 40, W, seeds, seed=21)
    levels, counts = oracle.segment(v, 26, 4)
    lv, c = ctx.segment(dev(v), 26, 4)
    ctx.check()
    assert c.cpu().tolist() == counts.tolist()
    assert np.array_equal(lv.cpu().numpy(), levels)


@pytest.mark.parametrize("W", [64, 72])
def test_segment_26_uint8_plateaux(ctx, W):
    v = (synth.distance_volume(24, 36, W, 15, seed=23) >> 10).astype(np.uint8)
    levels, counts = oracle.segment(v, 26, 3)
    lv, c = ctx.segment(dev(v), 26, 3)
    ctx.check()
    assert c.cpu().tolist() == counts.tolist()
    assert np.array_equal(lv.cpu().numpy(), levels)


def test_segment_batch_26(ctx):
    vols = [synth.distance_volume(d, h, w, n, seed=40 + i) for i, (d, h, w, n) in
            enumerate([(20, 30, 40, 12), (17, 33, 64, 200), (1, 1, 9, 1), (5, 70, 36, 40)])]
    levels, counts = ctx.segment_batch([dev(v) for v in vols], 26, 4)
    ctx.check()
    for v, lv, c in zip(vols, levels, counts):
        ref_l, ref_c = oracle.segment(v, 26, 4)
        assert c.cpu().tolist() == ref_c.tolist()
        assert np.array_equal(lv.cpu().numpy(), ref_l)


def test_static_26(ctx):
    from paper_2410_08946_gb300 import binding
    L = binding.load()
    P = ctypes.c_void_p
    L.ws_watershed_static.argtypes = [P, ctypes.c_int, ctypes.POINTER(binding.ws_shape), ctypes.c_int, P, P, P]
    L.ws_watershed_static.restype = ctypes.c_int
    v = synth.distance_volume(20, 24, 40, 30, seed=25)
    g = dev(v)
    labels = torch.full(g.shape, -7, dtype=torch.int32, device="cuda")
    count = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    sh = binding._shape_of(g.shape)
    st = L.ws_watershed_static(ctypes.c_void_p(g.data_ptr()), binding.WS_U16, ctypes.byref(sh), 26,
                               ctypes.c_void_p(labels.data_ptr()), ctypes.c_void_p(count.data_ptr()), None)
    assert st == binding.WS_OK
    torch.cuda.synchronize()
    ref, K = oracle.watershed(v, 26)
    assert int(count.cpu()[0]) == K
    assert np.array_equal(labels.cpu().numpy(), ref)
