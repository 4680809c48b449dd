"""The request loop (ws_server_*): requests of mixed kinds and sizes submitted
together are batched and overlapped on the device, and each result must be
exactly what ws_segment returns for that image alone (tolerance 0)."""
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


@pytest.fixture(scope="module")
def pool():
    g2 = oracle.gradient2d(synth.blob_image(600, 700, 120, seed=11))
    g3 = synth.distance_volume(48, 56, 64, 40, seed=12)
    return g2, g3


def _requests(pool, n, seed):
    """n (array, conn, NL) requests: 2D crops of the blob gradient (u8) and 3D
    crops of the distance volume (u16), sizes drawn at random."""
    g2, g3 = pool
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        if rng.random() < 0.7:
            h, w = (int(v) for v in rng.integers(1, 300, size=2))
            y, x = int(rng.integers(0, g2.shape[0] - h)), int(rng.integers(0, g2.shape[1] - w))
            out.append((np.ascontiguousarray(g2[y:y + h, x:x + w]), int(rng.choice([4, 8])), 4))
        else:
            d, h, w = (int(v) for v in rng.integers(2, 40, size=3))
            out.append((np.ascontiguousarray(g3[:d, :h, :w]), 6, 4))
    return out


def _reference(ctx, arr, conn, NL):
    lv, cnt = ctx.segment(torch.from_numpy(arr).cuda(), conn, NL)
    ctx.check()
    return lv.cpu(), cnt.cpu()


@pytest.mark.parametrize("on_host", [True, False])
def test_server_mix_matches_alone(ctx, pool, on_host):
    from paper_2410_08946_gb300 import binding
    reqs = _requests(pool, 60, seed=1 if on_host else 2)
    with binding.Server(0, budget_bytes=2 << 30, lanes=3, max_batch=16) as srv:
        tickets = []
        for arr, conn, NL in reqs:
            t = torch.from_numpy(arr)
            t = t.pin_memory() if on_host else t.cuda()
            tickets.append(srv.submit(t, conn, NL))
        for (arr, conn, NL), tk in zip(reqs, tickets):
            st, lv, cnt = srv.poll(tk, 120_000_000)
            assert st == binding.WS_OK
            ref_l, ref_c = _reference(ctx, arr, conn, NL)
            assert torch.equal(lv.cpu(), ref_l)
            assert torch.equal(cnt.cpu(), ref_c)


def test_server_against_oracle(ctx, pool):
    from paper_2410_08946_gb300 import binding
    arr = np.ascontiguousarray(pool[0][:200, :300])
    with binding.Server(0, lanes=2) as srv:
        tk = srv.submit(torch.from_numpy(arr).pin_memory(), 8, 5)
        st, lv, cnt = srv.poll(tk, 120_000_000)
    assert st == binding.WS_OK
    levels, counts = oracle.segment(arr, 8, 5)
    assert np.array_equal(lv.numpy(), levels) and cnt.tolist() == counts.tolist()


def test_server_cancel_and_budget(ctx, pool):
    from paper_2410_08946_gb300 import binding
    reqs = _requests(pool, 40, seed=3)
    with binding.Server(0, budget_bytes=1 << 30, lanes=1, max_batch=4) as srv:
        tickets = [srv.submit(torch.from_numpy(a).pin_memory(), c, nl) for a, c, nl in reqs]
        cancelled = [tk for tk in tickets[20:] if srv.cancel(tk) == binding.WS_OK]
        for (arr, conn, NL), tk in zip(reqs, tickets):
            st, lv, cnt = srv.poll(tk, 120_000_000)
            if tk in cancelled:
                assert st in (binding.WS_ERR_CANCELLED, binding.WS_OK)
            else:
                assert st == binding.WS_OK
                assert torch.equal(lv, _reference(ctx, arr, conn, NL)[0])
        # a request that alone exceeds a lane's share is refused at submit
        big = torch.zeros((8192, 8192), dtype=torch.uint8).pin_memory()
        with pytest.raises(binding.WsError) as e:
            srv.submit(big, 4, 6)
        assert e.value.status == binding.WS_ERR_OOM


def test_server_destroy_with_work_queued(ctx, pool):
    from paper_2410_08946_gb300 import binding
    reqs = _requests(pool, 30, seed=4)
    srv = binding.Server(0, lanes=1, max_batch=2)
    for a, c, nl in reqs:
        srv.submit(torch.from_numpy(a).cuda(), c, nl)
    srv.close()   # cancels what is queued, waits for what runs
