"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element, at sizes spanning several tiles with ragged tails.  Tolerance 0:
every stage is integer, so labels must be identical (both sides write
canonical labels)."""
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


def host(t):
    return t.cpu().numpy()


def rand_img(rng, shape, levels, dtype=np.uint8):
    return rng.integers(0, levels, size=shape).astype(dtype)


def blob_grad(H, W, seed, shift=0, blobs=None):
    img = synth.blob_image(H, W, blobs or synth.blob_count_for(H, W), seed)
    return oracle.gradient2d(img, shift)


CASES_2D = [((1, 1), 3), ((1, 37), 3), ((37, 1), 3), ((33, 65), 3), ((70, 45), 2), ((97, 131), 5),
            ((64, 64), 256)]
CASES_3D = [((1, 1, 1), 3), ((3, 17, 33), 3), ((9, 20, 18), 2), ((17, 9, 40), 4), ((10, 10, 10), 65536)]


# --------------------------------------------------------------------------
# step I
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,levels", CASES_2D)
@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_step1_2d(ctx, shape, levels, conn, dtype):
    rng = np.random.default_rng(hash((shape, levels, conn)) % 2**32)
    img = rand_img(rng, shape, min(levels, 256 if dtype == np.uint8 else 65536), dtype)
    S, L = oracle.step1(img, conn)
    s_d, l_d = ctx.step1(dev(img), conn)
    ctx.check()
    assert np.array_equal(host(s_d), S)
    assert np.array_equal(host(l_d), L)


@pytest.mark.parametrize("shape,levels", CASES_3D)
def test_step1_3d(ctx, shape, levels):
    rng = np.random.default_rng(11)
    img = rand_img(rng, shape, levels, np.uint16)
    S, L = oracle.step1(img, 6)
    s_d, l_d = ctx.step1(dev(img), 6)
    ctx.check()
    assert np.array_equal(host(s_d), S)
    assert np.array_equal(host(l_d), L)


# Step I runs in the segmentation path's own tiled kernels (k_init for 2D and
# 26-connectivity, k_init6 for 6-connectivity).  The shapes below give tiles
# whose halo lies inside the image (the branch-free interior code) beside
# border tiles, with rows that are 16-byte multiples (the gradient staged by
# TMA) and rows that are not (plain loads).
STEP1_TILES = [
    ((200, 256), 4, np.uint8, 3),      # 2D TMA (256 B rows), interior tiles
    ((200, 256), 8, np.uint16, 5),     # 2D TMA (512 B rows)
    ((130, 203), 4, np.uint8, 3),      # 2D plain loads (203 B rows)
    ((130, 203), 8, np.uint16, 256),
    ((50, 50, 96), 6, np.uint16, 4),   # 3D TMA (192 B rows), interior tiles
    ((50, 50, 96), 6, np.uint8, 2),    # 3D TMA (96 B rows)
    ((40, 40, 97), 6, np.uint16, 3),   # 3D plain loads
    ((40, 36, 96), 26, np.uint16, 3),  # 3D 26-connectivity, TMA
    ((20, 19, 37), 26, np.uint8, 2),   # 3D 26-connectivity, plain loads
]


@pytest.mark.parametrize("shape,conn,dtype,levels", STEP1_TILES)
def test_step1_tiled_kernels(ctx, shape, conn, dtype, levels):
    rng = np.random.default_rng(sum(shape) * conn + levels)
    img = rand_img(rng, shape, levels, dtype)
    S, L = oracle.step1(img, conn)
    s_d, l_d = ctx.step1(dev(img), conn)
    ctx.check()
    assert np.array_equal(host(s_d), S)
    assert np.array_equal(host(l_d), L)


def test_step1_distance_volume(ctx):
    """Step I of a distance-field volume (the benchmark's kind of input) with
    interior tiles on both staging paths."""
    for shape in ((48, 64, 128), (33, 47, 99)):
        vol = synth.distance_volume(*shape, 40, seed=sum(shape))
        S, L = oracle.step1(vol, 6)
        s_d, l_d = ctx.step1(dev(vol), 6)
        ctx.check()
        assert np.array_equal(host(s_d), S)
        assert np.array_equal(host(l_d), L)


# --------------------------------------------------------------------------
# step II distances
# --------------------------------------------------------------------------

@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("shape,levels", [((50, 70), 2), ((130, 97), 3), ((1, 300), 2), ((300, 1), 2)])
def test_plateau_distance_2d(ctx, conn, shape, levels):
    rng = np.random.default_rng(5)
    img = rand_img(rng, shape, levels)
    d_ref = oracle.plateau_distance(img, conn)
    d = host(ctx.plateau_distance(dev(img), conn))
    ctx.check()
    assert np.array_equal(d, d_ref)


@pytest.mark.parametrize("conn", [4, 8])
def test_plateau_distance_quantised_blobs(ctx, conn):
    g = blob_grad(300, 400, 77, shift=4)
    d_ref = oracle.plateau_distance(g, conn)
    d = host(ctx.plateau_distance(dev(g), conn))
    ctx.check()
    assert np.array_equal(d, d_ref)


def test_plateau_distance_long_snake(ctx):
    """A one-pixel-wide serpentine plateau that crosses many tiles back and forth."""
    H, W = 200, 210
    img = np.full((H, W), 9, dtype=np.uint8)
    for r in range(1, H - 1, 2):
        img[r, 1:W - 1] = 5
        if r + 1 < H - 1:
            c = W - 2 if (r // 2) % 2 == 0 else 1
            img[r + 1, c] = 5
    img[1, 1] = 4   # the exit at one end
    for conn in (4, 8):
        d_ref = oracle.plateau_distance(img, conn)
        d = host(ctx.plateau_distance(dev(img), conn))
        ctx.check()
        assert np.array_equal(d, d_ref)
        assert d_ref.max() > 5000


def test_plateau_distance_3d(ctx):
    rng = np.random.default_rng(6)
    img = rand_img(rng, (20, 30, 40), 2, np.uint16)
    d_ref = oracle.plateau_distance(img, 6)
    d = host(ctx.plateau_distance(dev(img), 6))
    ctx.check()
    assert np.array_equal(d, d_ref)


# --------------------------------------------------------------------------
# watershed
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,levels", CASES_2D + [((256, 256), 4), ((129, 200), 7)])
@pytest.mark.parametrize("conn", [4, 8])
def test_watershed_random_2d(ctx, shape, levels, conn):
    rng = np.random.default_rng(hash((shape, levels, conn, 1)) % 2**32)
    img = rand_img(rng, shape, levels)
    L, K = oracle.watershed(img, conn)
    l_d, k_d = ctx.watershed(dev(img), conn)
    ctx.check()
    assert int(host(k_d)[0]) == K
    assert np.array_equal(host(l_d), L)


@pytest.mark.parametrize("shape,levels", CASES_3D + [((33, 34, 35), 3)])
def test_watershed_random_3d(ctx, shape, levels):
    rng = np.random.default_rng(hash((shape, levels)) % 2**32)
    img = rand_img(rng, shape, levels, np.uint16)
    L, K = oracle.watershed(img, 6)
    l_d, k_d = ctx.watershed(dev(img), 6)
    ctx.check()
    assert int(host(k_d)[0]) == K
    assert np.array_equal(host(l_d), L)


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("shift", [0, 4])
def test_watershed_blobs_256(ctx, conn, shift):
    g = blob_grad(256, 256, synth.BASE_SEED, shift)
    L, K = oracle.watershed(g, conn)
    l_d, k_d = ctx.watershed(dev(g), conn)
    ctx.check()
    assert int(host(k_d)[0]) == K
    assert np.array_equal(host(l_d), L)


@pytest.mark.parametrize("shape", [(40, 50, 60), (24, 40, 64), (17, 33, 96)])
def test_watershed_distance_volume(ctx, shape):
    """W = 64 and 96 rows are 16-byte multiples (TMA staging); W = 60 is not
    (plain-load staging)."""
    v = synth.distance_volume(*shape, 30, seed=3)
    L, K = oracle.watershed(v, 6)
    l_d, k_d = ctx.watershed(dev(v), 6)
    ctx.check()
    assert int(host(k_d)[0]) == K
    assert np.array_equal(host(l_d), L)


def test_watershed_edge_cases(ctx):
    cases = [np.zeros((1, 1), np.uint8), np.full((40, 33), 255, np.uint8), np.full((5, 6), 65535, np.uint16),
             (np.indices((30, 31)).sum(0) % 2 * 9).astype(np.uint8),
             np.arange(64 * 70, dtype=np.uint16).reshape(64, 70)]
    for img in cases:
        for conn in (4, 8):
            L, K = oracle.watershed(img, conn)
            l_d, k_d = ctx.watershed(dev(img), conn)
            ctx.check()
            assert int(host(k_d)[0]) == K
            assert np.array_equal(host(l_d), L)


def test_watershed_deterministic(ctx):
    g = blob_grad(300, 300, 9, shift=4)
    ref = None
    for _ in range(10):
        l_d, _ = ctx.watershed(dev(g), 8)
        ctx.check()
        got = host(l_d)
        if ref is None:
            ref = got
        assert np.array_equal(got, ref)


# --------------------------------------------------------------------------
# waterfall / segment
# --------------------------------------------------------------------------

@pytest.mark.parametrize("conn", [4, 8])
def test_segment_blobs(ctx, conn):
    g = blob_grad(256, 256, synth.BASE_SEED)
    levels, counts = oracle.segment(g, conn, 4)
    lv_d, c_d = ctx.segment(dev(g), conn, 4)
    ctx.check()
    assert host(c_d).tolist() == counts.tolist()
    assert np.array_equal(host(lv_d), levels)


@pytest.mark.parametrize("seed", range(6))
def test_waterfall_random(ctx, seed):
    rng = np.random.default_rng(seed)
    img = rand_img(rng, (60, 77), 9)
    for conn in (4, 8):
        L0, K = oracle.watershed(img, conn)
        lv, cnt = oracle.waterfall(L0, img, conn, 5)
        lv_d, c_d = ctx.waterfall(dev(L0), dev(img), conn, 5)
        ctx.check()
        assert host(c_d).tolist() == cnt.tolist()
        assert np.array_equal(host(lv_d), lv)


@pytest.mark.parametrize("shape", [(30, 40, 50), (20, 35, 72)])
def test_segment_3d(ctx, shape):
    v = synth.distance_volume(*shape, 25, seed=8)
    levels, counts = oracle.segment(v, 6, 6)
    lv_d, c_d = ctx.segment(dev(v), 6, 6)
    ctx.check()
    assert host(c_d).tolist() == counts.tolist()
    assert np.array_equal(host(lv_d), levels)


def test_segment_nl1_and_single_region(ctx):
    img = np.full((20, 20), 3, np.uint8)
    lv_d, c_d = ctx.segment(dev(img), 4, 3)
    ctx.check()
    assert host(c_d).tolist() == [1, 1, 1]
    assert not host(lv_d).any()
    g = blob_grad(64, 64, 4)
    levels, counts = oracle.segment(g, 4, 1)
    lv_d, c_d = ctx.segment(dev(g), 4, 1)
    ctx.check()
    assert np.array_equal(host(lv_d), levels)


def test_segment_host_matches_device(ctx):
    g = blob_grad(200, 300, 12)
    lv_d, c_d = ctx.segment(dev(g), 4, 5)
    ctx.check()
    lh, ch = ctx.segment_host(torch.from_numpy(g), 4, 5)
    assert np.array_equal(lh.numpy(), host(lv_d))
    assert ch.tolist() == host(c_d).tolist()


# --------------------------------------------------------------------------
# gradient
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(1, 1), (1, 50), (50, 1), (37, 45), (256, 256), (300, 517)])
@pytest.mark.parametrize("shift", [0, 4])
def test_gradient(ctx, shape, shift):
    rng = np.random.default_rng(sum(shape))
    img = rng.integers(0, 256, size=shape).astype(np.uint8)
    ref = oracle.gradient2d(img, shift)
    got = host(ctx.gradient(dev(img), shift))
    assert np.array_equal(got, ref)


def test_gradient_blobs(ctx):
    img = synth.blob_image(256, 256, 32, synth.BASE_SEED)
    assert np.array_equal(host(ctx.gradient(dev(img))), oracle.gradient2d(img))


# --------------------------------------------------------------------------
# errors
# --------------------------------------------------------------------------

def test_invalid_arguments(ctx):
    from paper_2410_08946_gb300 import binding
    img = dev(np.zeros((8, 8), np.uint8))
    with pytest.raises(binding.WsError) as e:
        ctx.watershed(img, 6)
    assert e.value.status == binding.WS_ERR_INVALID
    v = dev(np.zeros((4, 4, 4), np.uint16))
    with pytest.raises(binding.WsError) as e:
        ctx.watershed(v, 8)          # a 2D connectivity on a volume
    assert e.value.status == binding.WS_ERR_INVALID
    with pytest.raises(binding.WsError) as e:
        ctx.watershed(img, 26)       # a 3D connectivity on an image
    assert e.value.status == binding.WS_ERR_INVALID
    with pytest.raises(binding.WsError):
        ctx.segment(img, 4, 0)


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("shape", [(256, 256), (130, 301)])
def test_segment_crowded_path_ends(ctx, conn, shape):
    """A checkerboard of 0 and 1 (plus a ramp on the ones): every 0 is a strict
    minimum (4-connectivity) or part of a diagonal plateau of minima
    (8-connectivity), so a tile's box holds more distinct path ends than the
    adjacency kernel's shared table; the ends it cannot list are chased one by
    one, and the labels stay those of the oracle."""
    H, W = shape
    yy, xx = np.mgrid[0:H, 0:W]
    img = (((yy + xx) % 2) * (1 + (xx * 7 + yy * 3) % 200)).astype(np.uint8)
    levels, counts = oracle.segment(img, conn, 3)
    lv_d, c_d = ctx.segment(dev(img), conn, 3)
    ctx.check()
    assert host(c_d).tolist() == counts.tolist()
    assert np.array_equal(host(lv_d), levels)


@pytest.mark.parametrize("conn", [4, 8])
def test_segment_plateau_terraces(ctx, conn):
    """Wide flat terraces (a blob gradient quantised to 4 levels): long plateau
    descents inside and across tiles, minimal plateaux joined across tile
    borders, tiles that are almost all plateau next to tiles with few plateau
    pixels."""
    g = blob_grad(300, 421, 21)
    img = (g >> 6).astype(np.uint8)
    levels, counts = oracle.segment(img, conn, 4)
    lv_d, c_d = ctx.segment(dev(img), conn, 4)
    ctx.check()
    assert host(c_d).tolist() == counts.tolist()
    assert np.array_equal(host(lv_d), levels)
