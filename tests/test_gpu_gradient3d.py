"""3D gradient (blur + Sobel magnitude of a volume) through the C ABI against
the oracle, voxel by voxel with tolerance 0 (integer arithmetic throughout),
and the 3D pipeline gradient -> watershed -> waterfall on its output."""
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


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (8, 8, 32), (9, 17, 33), (20, 30, 70), (5, 64, 100),
                                   (65, 17, 40), (128, 40, 31), (130, 9, 33)])   # several 64-plane chunks
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_random_volumes(ctx, shape, dtype):
    rng = np.random.default_rng(sum(shape))
    v = rng.integers(0, np.iinfo(dtype).max, size=shape, endpoint=True).astype(dtype)
    for shift in (0, 5):
        g = ctx.gradient3d(torch.from_numpy(v).cuda(), shift)
        ctx.check()
        assert np.array_equal(g.cpu().numpy(), oracle.gradient3d(v, shift))


def test_smooth_volume_and_pipeline(ctx):
    """A blob volume (smooth intensities, uint8), its gradient, then the 3D
    watershed + waterfall of that gradient, all against the oracle."""
    D, H, W = 24, 40, 48
    z, y, x = np.indices((D, H, W))
    rng = np.random.default_rng(4)
    v = np.zeros((D, H, W))
    for _ in range(12):
        c = rng.uniform([0, 0, 0], [D, H, W])
        v += rng.uniform(40, 120) * np.exp(-((z - c[0]) ** 2 + (y - c[1]) ** 2 + (x - c[2]) ** 2) /
                                           (2 * rng.uniform(3, 8) ** 2))
    v = np.clip(np.rint(v) + rng.integers(0, 8, size=v.shape), 0, 255).astype(np.uint8)
    g = ctx.gradient3d(torch.from_numpy(v).cuda())
    ref = oracle.gradient3d(v)
    assert np.array_equal(g.cpu().numpy(), ref)
    for conn in (6, 26):
        lv, c = ctx.segment(g, conn, 4)
        ctx.check()
        rl, rc = oracle.segment(ref, conn, 4)
        assert c.cpu().tolist() == rc.tolist()
        assert np.array_equal(lv.cpu().numpy(), rl)


def test_distance_volume_uint16(ctx):
    v = synth.distance_volume(16, 48, 64, 50, seed=3)
    g = ctx.gradient3d(torch.from_numpy(v).cuda(), 2)
    ctx.check()
    assert np.array_equal(g.cpu().numpy(), oracle.gradient3d(v, 2))


def test_invalid(ctx):
    from paper_2410_08946_gb300 import binding
    import ctypes
    img = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(TypeError):
        ctx.gradient3d(img)                                   # the binding wants a volume
    out = torch.zeros((16, 16), dtype=torch.uint16, device="cuda")
    sh = binding._shape_of(img.shape)                         # and so does the C ABI (ndim 2)
    st = ctx.lib.ws_gradient3d(ctx.handle, binding._dev(img), binding.WS_U8, ctypes.byref(sh), 0,
                               binding._dev(out), binding._stream(None))
    assert st == binding.WS_ERR_UNSUPPORTED
    vol = torch.zeros((4, 8, 8), dtype=torch.uint16, device="cuda")
    with pytest.raises(binding.WsError):
        ctx.gradient3d(vol, out=vol)                          # in place: overlap
    with pytest.raises(binding.WsError):
        ctx.gradient3d(vol, shift=40)
