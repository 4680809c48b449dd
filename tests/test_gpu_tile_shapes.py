"""The tile shapes of the 2D uint8 pipeline (ws_tuning.tile_shape: 0 = 64 x 32
pixels / 256 threads, 1 = 32 x 32 / 256, 2 = 128 x 16 / 256, 3 = 64 x 32 /
512) give the oracle's results, tolerance 0: step I, step II distances, the
segmentation of single images (rows that TMA stages and rows it cannot, ragged
tails, large plateaux) and of an uneven batch.  2D uint16 and 3D images keep
their one shape whatever the setting."""
import numpy as np
import pytest

import oracle
from paper_2410_08946_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [0, 1, 2, 3]


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


def _grad(H, W, seed, shift=0):
    return oracle.gradient2d(synth.blob_image(H, W, synth.blob_count_for(H, W), seed), shift)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("conn", [4, 8])
def test_segment_shapes(ctx, shape, conn):
    ctx.set_tuning(tile_shape=shape)
    try:
        for (H, W), shift, seed in (((200, 256), 0, 1), ((131, 203), 0, 2), ((300, 97), 4, 3), ((1, 77), 0, 4),
                                    ((64, 1), 0, 5)):
            g = _grad(H, W, seed, shift)
            lv, c = ctx.segment(torch.from_numpy(g).cuda(), conn, 4)
            ctx.check()
            ref, rc = oracle.segment(g, conn, 4)
            assert c.cpu().tolist() == rc.tolist()
            assert np.array_equal(lv.cpu().numpy(), ref), (H, W)
    finally:
        ctx.set_tuning()


@pytest.mark.parametrize("shape", SHAPES)
def test_step1_and_distances_shapes(ctx, shape):
    rng = np.random.default_rng(shape)
    ctx.set_tuning(tile_shape=shape)
    try:
        for (H, W), levels in (((150, 256), 3), ((97, 203), 2)):
            img = rng.integers(0, levels, size=(H, W)).astype(np.uint8)
            for conn in (4, 8):
                S, L = oracle.step1(img, conn)
                s_d, l_d = ctx.step1(torch.from_numpy(img).cuda(), conn)
                d_d = ctx.plateau_distance(torch.from_numpy(img).cuda(), conn)
                ctx.check()
                assert np.array_equal(s_d.cpu().numpy(), S)
                assert np.array_equal(l_d.cpu().numpy(), L)
                assert np.array_equal(d_d.cpu().numpy(), oracle.plateau_distance(img, conn))
    finally:
        ctx.set_tuning()


@pytest.mark.parametrize("shape", SHAPES)
def test_batch_shapes(ctx, shape):
    rng = np.random.default_rng(40 + shape)
    shapes = [(1, 1), (33, 65), (64, 64)] + [tuple(int(v) for v in rng.integers(20, 260, size=2)) for _ in range(9)]
    grads = [_grad(h, w, 600 + i) for i, (h, w) in enumerate(shapes)]
    ctx.set_tuning(tile_shape=shape)
    try:
        levels, counts = ctx.segment_batch([torch.from_numpy(g).cuda() for g in grads], 4, 5)
        ctx.check()
    finally:
        ctx.set_tuning()
    for g, lv, c in zip(grads, levels, counts):
        ref, rc = oracle.segment(g, 4, 5)
        assert c.cpu().tolist() == rc.tolist()
        assert np.array_equal(lv.cpu().numpy(), ref)


def test_fixed_shape_images_ignore_the_setting(ctx):
    g16 = (_grad(90, 130, 7).astype(np.uint16) * 300)
    v = synth.distance_volume(20, 24, 40, 9, seed=8)
    ctx.set_tuning(tile_shape=2)
    try:
        lv, c = ctx.segment(torch.from_numpy(g16).cuda(), 8, 3)
        lv3, c3 = ctx.segment(torch.from_numpy(v).cuda(), 6, 3)
        ctx.check()
    finally:
        ctx.set_tuning()
    assert np.array_equal(lv.cpu().numpy(), oracle.segment(g16, 8, 3)[0])
    assert np.array_equal(lv3.cpu().numpy(), oracle.segment(v, 6, 3)[0])


def test_invalid_shape(ctx):
    from paper_2410_08946_gb300 import binding
    with pytest.raises(binding.WsError):
        ctx.set_tuning(tile_shape=4)
    ctx.set_tuning()
