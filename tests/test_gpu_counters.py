"""ws_context_counters: the device's counts of the last call agree with what
the oracle says of the same input (basins = K0, plateau pixels = the pixels
Eq. 1 puts in states 2 and 3), and the round counts are positive."""
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


@pytest.mark.parametrize("conn", [4, 8])
def test_counters_2d(ctx, conn):
    g = oracle.gradient2d(synth.blob_image(300, 400, 40, seed=21), 3)
    lv, cnt = ctx.segment(torch.from_numpy(g).cuda(), conn, 3)
    c = ctx.counters()
    S, _ = oracle.step1(g, conn)
    assert c["basins"] == int(cnt[0]) == oracle.watershed(g, conn)[1]
    assert c["plateau_pixels"] == int(np.isin(S, (2, 3)).sum())
    assert c["plateau_rounds"] >= 1 and c["jump_rounds"] >= 1
    assert c["plateau_tiles"] >= 1 and c["edge_records"] >= c["basins"] - 1


def test_counters_3d(ctx):
    v = synth.distance_volume(40, 48, 96, 30, seed=22)
    lv, cnt = ctx.segment(torch.from_numpy(v).cuda(), 6, 3)
    c = ctx.counters()
    assert c["basins"] == int(cnt[0]) == oracle.watershed(v, 6)[1]
    # every basin's root is an in-tile path end, and so is every voxel whose arrow leaves its tile
    assert c["path_ends"] >= c["basins"]
    assert c["edge_records"] >= 1
