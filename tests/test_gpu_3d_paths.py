"""3D path coverage: the per-tile regimes of the 3D labelling pass (basins per
tile within the 64-basin pass matrix, up to 253 ids with the shared edge
hash, beyond that the per-voxel root path), uint8 volumes with plateaux, both
staging paths (TMA needs rows of 16-byte multiples), and batches of 3D
volumes.  Tolerance 0 against the oracle (every stage is integer).

Each regime test first checks on the CPU, from the oracle's labels, that its
input really has the basin counts per tile it is meant to exercise."""
import numpy as np
import pytest

import oracle
from paper_2410_08946_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TX, TY, TZ = 32, 16, 16   # 3D tile (x, y, z)


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


def tile_basins(L):
    """Distinct basins per tile, counting the tile's +x, +y, +z face voxels."""
    D, H, W = L.shape
    out = []
    for z0 in range(0, D, TZ):
        for y0 in range(0, H, TY):
            for x0 in range(0, W, TX):
                s = set(np.unique(L[z0:z0 + TZ, y0:y0 + TY, x0:x0 + TX]).tolist())
                if z0 + TZ < D:
                    s |= set(np.unique(L[z0 + TZ, y0:y0 + TY, x0:x0 + TX]).tolist())
                if y0 + TY < H:
                    s |= set(np.unique(L[z0:z0 + TZ, y0 + TY, x0:x0 + TX]).tolist())
                if x0 + TX < W:
                    s |= set(np.unique(L[z0:z0 + TZ, y0:y0 + TY, x0 + TX]).tolist())
                out.append(len(s))
    return np.array(out)


def check_segment(ctx, v, NL):
    levels, counts = oracle.segment(v, 6, NL)
    lv, c = ctx.segment(torch.from_numpy(v).cuda(), 6, NL)
    ctx.check()
    assert c.cpu().tolist() == counts.tolist()
    assert np.array_equal(lv.cpu().numpy(), levels)


# (seeds, lowest and highest basins per tile the input must reach)
REGIMES = {
    "matrix": (30, 1, 64),          # every tile within the 64x64 pass matrix
    "mixed": (400, 50, 80),         # tiles on both sides of 64
    "hash": (1500, 65, 253),        # every tile in the shared-edge-hash regime
    "roots": (3000, 254, 10 ** 6),  # every tile beyond 253 ids
    "full": (6000, 254, 10 ** 6),   # beyond 253 ids, some tiles beyond the 512-slot basin hash
}


@pytest.mark.parametrize("regime", list(REGIMES))
@pytest.mark.parametrize("W", [64, 60])
def test_segment_3d_tile_regimes(ctx, regime, W):
    seeds, lo, hi = REGIMES[regime]
    v = synth.distance_volume(32, 48, W, seeds, seed=7)
    L, _ = oracle.watershed(v, 6)
    tb = tile_basins(L.reshape(v.shape))
    if regime == "mixed":
        assert tb.min() <= 64 < tb.max()
    elif regime == "full":
        assert tb.min() >= lo and tb.max() > 512, (tb.min(), tb.max())
    else:
        assert lo <= tb.min() and tb.max() <= hi, (tb.min(), tb.max())
    check_segment(ctx, v, 4)


@pytest.mark.parametrize("W", [64, 72])
def test_segment_3d_uint8_plateaux(ctx, W):
    """uint8 quantisation of a distance volume: large 3D plateaux (step II on
    plateau tiles); W = 64 takes the TMA staging, W = 72 the plain loads."""
    v = (synth.distance_volume(24, 40, W, 20, seed=11) >> 10).astype(np.uint8)
    assert len(np.unique(v)) < 70
    check_segment(ctx, v, 3)


def test_segment_3d_ragged_small(ctx):
    """Volumes smaller than one tile in every direction, and one voxel thick."""
    for shape in [(1, 1, 1), (1, 1, 50), (3, 5, 7), (17, 1, 33), (1, 17, 40), (16, 16, 32), (17, 17, 33)]:
        v = synth.distance_volume(*shape, 3, seed=sum(shape)) if min(shape) > 1 else \
            np.random.default_rng(sum(shape)).integers(0, 5, size=shape).astype(np.uint16)
        check_segment(ctx, v, 3)


def test_segment_batch_3d(ctx):
    """A batch of uneven 3D volumes (plain-load staging, tiles of several
    images in one launch, ends chased across the concatenated volumes)."""
    vols = [synth.distance_volume(d, h, w, n, seed=30 + i) for i, (d, h, w, n) in
            enumerate([(20, 30, 40, 12), (33, 17, 64, 300), (5, 70, 36, 40), (40, 40, 40, 1500), (1, 1, 9, 1)])]
    grads = [torch.from_numpy(v).cuda() for v in vols]
    levels, counts = ctx.segment_batch(grads, 6, 4)
    ctx.check()
    for v, lv, c in zip(vols, levels, counts):
        ref_l, ref_c = oracle.segment(v, 6, 4)
        assert c.cpu().tolist() == ref_c.tolist()
        assert np.array_equal(lv.cpu().numpy(), ref_l)
