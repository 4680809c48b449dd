"""Batched watershed + waterfall (ws_segment_batch) and its CUDA-graph replay
(ws_graph_create / ws_graph_launch): every image's result must be exactly
what ws_segment returns for it alone (tolerance 0), and what the oracle
computes."""
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


def _blob_grads(shapes, seed, shift=0):
    out = []
    for i, (h, w) in enumerate(shapes):
        img = synth.blob_image(h, w, synth.blob_count_for(h, w), seed + i)
        out.append(torch.from_numpy(oracle.gradient2d(img, shift)).cuda())
    return out


def _check_against_single(ctx, grads, conn, NL, levels, counts):
    for g, lv, cnt in zip(grads, levels, counts):
        ref_l, ref_c = ctx.segment(g, conn, NL)
        ctx.check()
        assert cnt.tolist() == ref_c.tolist()
        assert torch.equal(lv, ref_l)


@pytest.mark.parametrize("conn", [4, 8])
def test_batch_2d_uneven(ctx, conn):
    rng = np.random.default_rng(conn)
    shapes = [(1, 1), (1, 37), (45, 1), (64, 64), (33, 130)] + \
             [tuple(int(v) for v in rng.integers(20, 300, size=2)) for _ in range(10)]
    grads = _blob_grads(shapes, 100)
    levels, counts = ctx.segment_batch(grads, conn, 4)
    ctx.check()
    _check_against_single(ctx, grads, conn, 4, levels, counts)
    # one image against the oracle directly
    ref, rc = oracle.segment(grads[6].cpu().numpy(), conn, 4)
    assert np.array_equal(levels[6].cpu().numpy(), ref)


def test_batch_quantised_plateaux(ctx):
    shapes = [(120, 200), (300, 90), (64, 640), (256, 256)]
    grads = _blob_grads(shapes, 200, shift=4)
    levels, counts = ctx.segment_batch(grads, 8, 3)
    ctx.check()
    _check_against_single(ctx, grads, 8, 3, levels, counts)


def test_batch_3d(ctx):
    shapes = [(20, 30, 40), (17, 9, 64), (8, 8, 8), (1, 1, 5), (24, 40, 48)]
    grads = [torch.from_numpy(synth.distance_volume(*s, 12, seed=300 + i)).cuda() for i, s in enumerate(shapes)]
    levels, counts = ctx.segment_batch(grads, 6, 6)
    ctx.check()
    _check_against_single(ctx, grads, 6, 6, levels, counts)


def test_batch_nl1(ctx):
    grads = _blob_grads([(50, 60), (70, 10)], 400)
    levels, counts = ctx.segment_batch(grads, 4, 1)
    ctx.check()
    _check_against_single(ctx, grads, 4, 1, levels, counts)


def test_graph_replay(ctx):
    from paper_2410_08946_gb300 import binding
    rng = np.random.default_rng(7)
    shapes = [tuple(int(v) for v in rng.integers(30, 400, size=2)) for _ in range(24)]
    grads = _blob_grads(shapes, 500)
    g = ctx.graph(grads, 4, 6)
    ctx.check()
    eager = [lv.clone() for lv in g.levels]
    eager_c = [c.clone() for c in g.counts]
    for _ in range(2):
        for lv in g.levels:
            lv.fill_(-5)
        g.launch()
        ctx.check()
        for lv, ref in zip(g.levels, eager):
            assert torch.equal(lv, ref)
        for cnt, ref in zip(g.counts, eager_c):
            assert torch.equal(cnt, ref)
    _check_against_single(ctx, grads[:4], 4, 6, g.levels[:4], g.counts[:4])
    # growing the context's workspace invalidates the recorded graph
    big = torch.from_numpy(synth.distance_volume(160, 160, 160, 20, seed=1)).cuda()   # more pixels than the batch
    ctx.segment(big, 6, 6)
    ctx.check()
    with pytest.raises(binding.WsError) as e:
        g.launch()
    assert e.value.status == binding.WS_ERR_INVALID
    g.close()


def test_batch_invalid(ctx):
    from paper_2410_08946_gb300 import binding
    a = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    b = torch.zeros((4, 4, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(binding.WsError):
        ctx.segment_batch([a, b], 4, 2)
    with pytest.raises((binding.WsError, TypeError)):
        ctx.segment_batch([a, torch.zeros((8, 8), dtype=torch.uint16, device="cuda")], 4, 2)


def test_autotune_batch(ctx, tmp_path):
    """The autotuner times the batch under each candidate, leaves the fastest
    set on the context, caches it, and no parameter changes a label: the tuned
    batch equals the batch under the defaults and the oracle."""
    from paper_2410_08946_gb300 import autotune
    rng = np.random.default_rng(11)
    shapes = [tuple(int(v) for v in rng.integers(40, 400, size=2)) for _ in range(12)]
    grads = _blob_grads(shapes, 500, shift=2)
    ctx.set_tuning()
    ref_levels, ref_counts = ctx.segment_batch(grads, 4, 4)
    ctx.check()
    lv = [torch.empty_like(x) for x in ref_levels]
    ct = [torch.empty_like(x) for x in ref_counts]
    space = {"tile_shape": [0, 1, 2, 3], "jumps_per_round": [1, 3, 6], "levels_ctas_per_sm": [1, 4]}
    cache = str(tmp_path / "tune.json")
    res = autotune.autotune(ctx, lambda: ctx.segment_batch(grads, 4, 4, lv, ct), key="test", reps=2,
                            space=space, cache_path=cache)
    assert not res["cached"] and len(res["table"]) == 9
    assert res["params"]["jumps_per_round"] in (1, 3, 6) and res["params"]["levels_ctas_per_sm"] in (1, 4)
    assert res["params"]["tile_shape"] in (0, 1, 2, 3)
    for a, b in zip(lv, ref_levels):
        assert torch.equal(a, b)
    for a, b in zip(ct, ref_counts):
        assert torch.equal(a, b)
    # every candidate gives the same labels (every tile shape, jumps_per_round 1 and one CTA per SM included)
    for p in ({"jumps_per_round": 1, "levels_ctas_per_sm": 1}, {"jumps_per_round": 16, "levels_ctas_per_sm": 8},
              {"tile_shape": 1}, {"tile_shape": 2}, {"tile_shape": 3, "jumps_per_round": 1}):
        ctx.set_tuning(**p)
        levels, counts = ctx.segment_batch(grads, 4, 4)
        ctx.check()
        assert all(torch.equal(a, b) for a, b in zip(levels, ref_levels))
    again = autotune.autotune(ctx, lambda: None, key="test", cache_path=cache)
    assert again["cached"] and again["params"] == res["params"]
    ref, _ = oracle.segment(grads[3].cpu().numpy(), 4, 4)
    assert np.array_equal(ref_levels[3].cpu().numpy(), ref)
    ctx.set_tuning()
