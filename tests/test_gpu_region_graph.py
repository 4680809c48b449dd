"""Region-graph export (Sec. 6 graph of waterfall regions, Alg. 5 step V pass
values) through the C ABI against the oracle, element by element with
tolerance 0: CSR row starts, neighbour ids, pass values, region sizes, value
sums and the float64 means (sum / size, one correctly rounded division on both
sides).  Labellings come from the oracle's segmentation or from seeded
generators; none comes from the CUDA path."""
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


def compare(ctx, L, g, conn, values=None):
    ref = oracle.region_graph(L, g, conn, values=values)
    vt = None if values is None else torch.from_numpy(np.ascontiguousarray(values)).cuda()
    got = ctx.region_graph(torch.from_numpy(np.ascontiguousarray(L, dtype=np.int32)).cuda(),
                           torch.from_numpy(np.ascontiguousarray(g)).cuda(), conn, values=vt)
    ctx.check()
    assert got["row_ptr"].cpu().numpy().tolist() == ref["row_ptr"].tolist()
    assert np.array_equal(got["col"].cpu().numpy(), ref["col"])
    assert np.array_equal(got["pass"].cpu().numpy().astype(np.uint32), ref["pass"])
    assert np.array_equal(got["size"].cpu().numpy(), ref["size"])
    assert np.array_equal(got["sum"].cpu().numpy().astype(np.uint64), ref["sum"])
    assert np.array_equal(got["mean"].cpu().numpy(), ref["mean"])
    return ref


@pytest.mark.parametrize("conn", [4, 8])
def test_fragmented_2d_levels(ctx, conn):
    """A noise gradient (thousands of basins, entries over many 4096-key radix
    tiles) with a ragged size; every level of a 4-level waterfall, 3 uint16
    value channels."""
    rng = np.random.default_rng(5 + conn)
    g = rng.integers(0, 256, size=(203, 317)).astype(np.uint8)
    levels, counts = oracle.segment(g, conn, 4)
    assert counts[0] > 5000
    vals = rng.integers(0, 65536, size=(3, 203, 317)).astype(np.uint16)
    for k in range(4):
        ref = compare(ctx, levels[k], g, conn, vals)
        assert len(ref["row_ptr"]) == counts[k] + 1


@pytest.mark.parametrize("conn", [6, 26])
def test_volume_levels(ctx, conn):
    v = synth.distance_volume(24, 40, 60, 900, seed=4)
    levels, counts = oracle.segment(v, conn, 3)
    vals = (v >> 4).astype(np.uint8)
    for k in range(3):
        compare(ctx, levels[k], v, conn, vals)


@pytest.mark.parametrize("conn", [4, 8])
def test_uint16_distance_image(ctx, conn):
    v = synth.distance_volume(1, 512, 384, 2000, seed=8)[0]
    levels, _ = oracle.segment(v, conn, 2)
    compare(ctx, levels[0], v, conn)
    compare(ctx, levels[1], v, conn, v)


def test_all_distinct_ids(ctx):
    """K = N (every pixel its own region): 20-bit ids, 40-bit keys, an odd
    number (5) of radix passes; random permutation of the ids."""
    rng = np.random.default_rng(1)
    H, W = 256, 300
    L = rng.permutation(H * W).astype(np.int32).reshape(H, W)
    g = rng.integers(0, 65536, size=(H, W)).astype(np.uint16)
    compare(ctx, L, g, 8, g)


def test_gaps_and_small_cases(ctx):
    rng = np.random.default_rng(2)
    # ids with gaps (sizes 0, means 0)
    L = (rng.integers(0, 7, size=(33, 41)) * 3).astype(np.int32)
    g = rng.integers(0, 256, size=(33, 41)).astype(np.uint8)
    compare(ctx, L, g, 4, g)
    # one region: no edge
    compare(ctx, np.zeros((17, 9), np.int32), g[:17, :9], 8, g[:17, :9])
    # one pixel
    compare(ctx, np.zeros((1, 1), np.int32), g[:1, :1], 4)
    # two regions (one radix pass), thin volume
    L3 = np.zeros((1, 5, 70), np.int32)
    L3[..., 35:] = 1
    compare(ctx, L3, rng.integers(0, 9, size=(1, 5, 70)).astype(np.uint8), 26)


def test_random_blocks_3d(ctx):
    """Axis-aligned random blocks with random ids (many regions per tile,
    diagonal-only contacts for 26-connectivity)."""
    rng = np.random.default_rng(3)
    D, H, W = 20, 26, 35
    z, y, x = np.indices((D, H, W))
    L = ((z // 3) * 100 + (y // 4) * 10 + (x // 5)).astype(np.int32)
    perm = rng.permutation(int(L.max()) + 1).astype(np.int32)
    L = perm[L]
    g = rng.integers(0, 1000, size=(D, H, W)).astype(np.uint16)
    for conn in (6, 26):
        compare(ctx, L, g, conn, np.stack([g, g // 3]).astype(np.uint16))


def test_deterministic(ctx):
    rng = np.random.default_rng(4)
    g = torch.from_numpy(rng.integers(0, 256, size=(300, 300)).astype(np.uint8)).cuda()
    L = torch.from_numpy(oracle.watershed(g.cpu().numpy(), 8)[0]).cuda()
    a = ctx.region_graph(L, g, 8)
    b = ctx.region_graph(L, g, 8)
    for key in ("row_ptr", "col", "pass", "size"):
        assert torch.equal(a[key], b[key])


def test_invalid_labels(ctx):
    from paper_2410_08946_gb300 import binding
    g = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    L = torch.zeros((8, 8), dtype=torch.int32, device="cuda")
    L[3, 3] = -1
    with pytest.raises(binding.WsError) as e:
        ctx.region_graph(L, g, 4)
    assert e.value.status == binding.WS_ERR_INVALID
    L[3, 3] = 64   # not below the pixel count
    with pytest.raises(binding.WsError):
        ctx.region_graph(L, g, 4)
    L[3, 3] = 2 ** 31 - 1
    with pytest.raises(binding.WsError):
        ctx.region_graph(L, g, 4)
    L[3, 3] = 63
    ctx.region_graph(L, g, 4)
    with pytest.raises(binding.WsError):
        ctx.region_graph(L, g, 6)   # 3D connectivity on an image
    fresh = binding.Context(0)
    try:
        st = fresh.lib.ws_region_graph_read(fresh.handle, None, None, None, None, None, None, None)
        assert st == binding.WS_ERR_INVALID
    finally:
        fresh.close()


@pytest.mark.parametrize("shape,conn,dt", [((37, 128), 4, np.uint8), ((41, 64), 4, np.uint16),
                                           ((9, 13, 64), 6, np.uint8), ((7, 11, 36), 6, np.uint16)])
def test_aligned_widths_and_offset_view(ctx, shape, conn, dt):
    """Widths that are multiples of 4 (u8 and u16 heights, 2D and 3D), and the
    same labelling starting 4 bytes past an aligned address (a contiguous view
    the library must not assume to be 16-byte aligned).  Both against the
    oracle."""
    rng = np.random.default_rng(sum(shape))
    g = rng.integers(0, 200 if dt == np.uint8 else 50000, size=shape).astype(dt)
    L, _ = oracle.watershed(g, conn)
    compare(ctx, L, g, conn, g)
    buf = torch.empty(L.size + 1, dtype=torch.int32, device="cuda")
    buf[1:] = torch.from_numpy(L.ravel()).cuda()
    Lm = buf[1:].view(shape)                      # contiguous, 4 bytes off a 16-byte boundary
    got = ctx.region_graph(Lm, torch.from_numpy(g).cuda(), conn)
    ctx.check()
    ref = oracle.region_graph(L, g, conn)
    assert np.array_equal(got["col"].cpu().numpy(), ref["col"])
    assert np.array_equal(got["pass"].cpu().numpy().astype(np.uint32), ref["pass"])
    assert got["row_ptr"].cpu().numpy().tolist() == ref["row_ptr"].tolist()
