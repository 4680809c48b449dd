"""Failure detection without a GPU fault.  Every device loop of the library is
bounded; when a bound runs out the kernel records an error in the context's
status word and returns, and ws_context_check reports it.  These tests make
bounds run out on purpose through ws_tuning -- a step II round cap, a pointer
jumping round cap, a region table too small for the image, a device-wide
barrier whose wait runs out because one block withholds its arrival -- check
the status the host reads, and then check that the same context computes the
same input correctly once the tuning is back to its defaults (the context
stays usable; nothing traps, faults or hangs)."""
import numpy as np
import pytest

import oracle
from paper_2410_08946_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_08946_gb300 import binding
    c = binding.Context(0)
    yield c
    c.close()


def _expect(ctx, status, fn):
    from paper_2410_08946_gb300 import binding
    fn()
    with pytest.raises(binding.WsError) as e:
        ctx.check()
    assert e.value.status == status, str(e.value)
    ctx.check()   # the status word was cleared by the report


def _parity(ctx, g, conn, NL):
    lv, c = ctx.segment(torch.from_numpy(g).cuda(), conn, NL)
    ctx.check()
    ref_l, ref_c = oracle.segment(g, conn, NL)
    assert c.cpu().tolist() == ref_c.tolist()
    assert np.array_equal(lv.cpu().numpy(), ref_l)


def test_plateau_round_cap(ctx):
    """A plateau 600 pixels long whose only lower border is at one end: its
    step II distances cross about ten tiles, one device-wide round each."""
    from paper_2410_08946_gb300 import binding
    g = np.full((40, 600), 9, dtype=np.uint8)
    g[:, 0] = 3
    g[:, 1:] = 7
    g[5:35, 20:580] = 7
    g[0, :] = 9
    g[-1, :] = 9
    ctx.set_tuning(plateau_round_cap=1)
    _expect(ctx, binding.WS_ERR_NONCONVERGED, lambda: ctx.segment(torch.from_numpy(g).cuda(), 4, 3))
    ctx.set_tuning()
    _parity(ctx, g, 4, 3)


def test_jump_round_cap(ctx):
    """A one-pixel-wide serpentine plateau: its paths cross tiles hundreds of
    times, so one jump per round cannot finish in one round."""
    from paper_2410_08946_gb300 import binding
    H, W = 64, 256
    g = np.full((H, W), 50, dtype=np.uint8)
    for r in range(1, H - 1, 2):
        g[r, 1:W - 1] = 10                            # corridors
        g[r + 1, (W - 2) if (r // 2) % 2 == 0 else 1] = 10   # alternate turns
    g[1, 1] = 5                                       # the one exit, at the start of the corridor
    ctx.set_tuning(jump_round_cap=1, jumps_per_round=1)
    _expect(ctx, binding.WS_ERR_NONCONVERGED, lambda: ctx.segment(torch.from_numpy(g).cuda(), 4, 2))
    ctx.set_tuning()
    _parity(ctx, g, 4, 2)


def test_region_table_full():
    """A noise image (52,433 basins, 140,699 adjacent pairs) against the
    smallest region table (65,536 slots): inserts give up after their probe
    limit and the call reports WS_ERR_OOM; a context with the default table
    then gets it right."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_08946_gb300 import binding
    g = np.random.default_rng(4).integers(0, 256, size=(512, 512)).astype(np.uint8)
    small = binding.Context(0)
    try:
        small.set_tuning(edge_capacity=65536)
        _expect(small, binding.WS_ERR_OOM, lambda: small.segment(torch.from_numpy(g).cuda(), 4, 3))
    finally:
        small.close()
    fresh = binding.Context(0)
    try:
        _parity(fresh, g, 4, 3)
    finally:
        fresh.close()


def _plateau_image():
    g = np.full((40, 600), 9, dtype=np.uint8)
    g[:, 0] = 3
    g[:, 1:] = 7
    g[5:35, 20:580] = 7
    g[0, :] = 9
    g[-1, :] = 9
    return g


@pytest.mark.parametrize("kind", ["segment2d", "segment3d", "waterfall"])
def test_barrier_timeout(ctx, kind):
    """A device-wide barrier wait that runs out.  With ws_tuning's one-shot
    barrier_withhold armed, block 0 of the next cooperative kernel (the step II
    relaxation of a segmentation; the level kernel of a waterfall over given
    labels) does not arrive at its first barrier, so the other blocks' waits
    run out after barrier_timeout_ms = 1: the call ends within a fraction of
    the default 4 s limit, ws_context_check reports WS_ERR_TIMEOUT, and the
    same context then computes the same input correctly."""
    import time
    from paper_2410_08946_gb300 import binding
    if kind == "segment3d":
        g, conn = synth.distance_volume(40, 48, 96, 30, seed=77), 6
    else:
        g, conn = _plateau_image(), 4
    g_d = torch.from_numpy(g).cuda()
    if kind == "waterfall":
        l0 = torch.from_numpy(oracle.watershed(g, conn)[0]).cuda()
        run = lambda: ctx.waterfall(l0, g_d, conn, 4)   # noqa: E731
    else:
        run = lambda: ctx.segment(g_d, conn, 3)          # noqa: E731
    run()            # workspace allocated, nothing armed
    ctx.check()
    ctx.set_tuning(barrier_timeout_ms=1, barrier_withhold=1)
    t0 = time.perf_counter()
    _expect(ctx, binding.WS_ERR_TIMEOUT, run)
    assert time.perf_counter() - t0 < 2.0, "a barrier wait did not end at its limit"
    ctx.set_tuning()
    if kind == "waterfall":
        ref_l, ref_c = oracle.waterfall(l0.cpu().numpy(), g, conn, 4)
        lv, c = ctx.waterfall(l0, g_d, conn, 4)
        ctx.check()
        assert c.cpu().tolist() == ref_c.tolist()
        assert np.array_equal(lv.cpu().numpy(), ref_l)
    else:
        _parity(ctx, g, conn, 3)


def test_barrier_withhold_is_one_shot(ctx):
    """The hold goes to one launch only: the next call on the context, with
    the same tuning left in place, completes without error."""
    from paper_2410_08946_gb300 import binding
    g = _plateau_image()
    g_d = torch.from_numpy(g).cuda()
    ctx.set_tuning(barrier_timeout_ms=50, barrier_withhold=1)
    _expect(ctx, binding.WS_ERR_TIMEOUT, lambda: ctx.segment(g_d, 4, 3))
    _parity(ctx, g, 4, 3)
    with pytest.raises(binding.WsError):
        ctx.set_tuning(barrier_withhold=2)
    ctx.set_tuning()
