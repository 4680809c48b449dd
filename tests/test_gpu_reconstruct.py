"""Paper-literal waterfall (Alg. 4 with the image reconstruction of Alg. 5)
through the C ABI against the oracle, every level plane and count with
tolerance 0.  Raising each basin to its lowest pass creates large plateaux,
so the levels above 0 exercise step II and step IV heavily."""
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


def check(ctx, g, conn, NL):
    ref_l, ref_c = oracle.waterfall_reconstruct(g, conn, NL)
    lv, c = ctx.waterfall_reconstruct(torch.from_numpy(np.ascontiguousarray(g)).cuda(), conn, NL)
    ctx.check()
    assert c.cpu().tolist() == ref_c.tolist()
    assert np.array_equal(lv.cpu().numpy(), ref_l)
    return ref_c


def test_hand_derived_1d(ctx):
    g = np.array([[10, 100, 50, 200, 80, 90, 5]], dtype=np.uint8)
    c = check(ctx, g, 4, 3)
    assert c.tolist() == [4, 2, 1]


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_2d(ctx, conn, dtype):
    v = synth.distance_volume(1, 300, 257, 400, seed=12)[0]
    g = v.astype(np.uint16) if dtype == np.uint16 else (v >> 6).astype(np.uint8)
    c = check(ctx, g, conn, 5)
    assert c[0] > 100


def test_2d_noise_uint8(ctx):
    """A noise image (a basin every few pixels): many small raised plateaux."""
    rng = np.random.default_rng(3)
    g = rng.integers(0, 256, size=(130, 190)).astype(np.uint8)
    check(ctx, g, 8, 6)


@pytest.mark.parametrize("conn", [6, 26])
def test_3d(ctx, conn):
    v = synth.distance_volume(30, 40, 64, 600, seed=13)
    check(ctx, v, conn, 4)


def test_3d_ragged_and_plain_loads(ctx):
    """Widths whose rows are not 16-byte multiples (plain-load staging), and
    volumes thinner than a tile."""
    for shape in [(17, 21, 45), (3, 40, 70), (1, 1, 33)]:
        v = synth.distance_volume(*shape, 25, seed=sum(shape)) if min(shape) > 1 else \
            np.random.default_rng(1).integers(0, 9, size=shape).astype(np.uint16)
        check(ctx, v, 6, 4)


def test_single_level_is_the_watershed(ctx):
    v = synth.distance_volume(1, 64, 96, 30, seed=2)[0]
    lv, c = ctx.waterfall_reconstruct(torch.from_numpy(v).cuda(), 4, 1)
    ctx.check()
    L, K = oracle.watershed(v, 4)
    assert c.cpu().tolist() == [K] and np.array_equal(lv[0].cpu().numpy(), L)
