"""Full-size workloads, in the launch configuration bench.py times, against
the oracle:

  2D 256 x 256 uint8 blob image, GPU gradient, 4-connectivity, NL = 3
  2D 4096 x 4096 uint8 blob gradient quantised to 16 levels (>> 4), 4- and
     8-connectivity, NL = 6 (large plateaux)
  3D 928 x 928 x 928 uint16 distance-field volume, 6-connectivity, NL = 6:
     every label plane element by element (the oracle takes about two and a
     half minutes on one host core), and properties that hold at any size
     (canonical ids, nesting, counts, one minimal plateau per basin with the
     plateaux found by an independent connected-component labelling)
  the 512-image batch (2D uint8 crops with sides log-uniform in [64, 2048] of
     a 4096^2 blob gradient, 4-connectivity, NL = 6) as one CUDA-graph replay:
     every image against the oracle
  a served mix shaped like the request stream (80% 2D uint8 crops with sides
     in [256, 4096], 20% 3D uint16 crops with sides in [64, 256], NL = 4)
     submitted at once to a four-lane server: every result against the oracle

The many-image cases run the oracle in spawned worker processes and compare
SHA-256 digests of the whole label planes (and the region counts); an image
whose digests differ is recomputed in-process and reported element by element.
"""
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


def test_blob_256_full_pipeline(ctx):
    img = synth.blob_image(256, 256, 32, synth.BASE_SEED + 0)
    img_d = torch.from_numpy(img).cuda()
    grad_d = ctx.gradient(img_d)
    lv_d, c_d = ctx.segment(grad_d, 4, 3)
    ctx.check()
    grad = oracle.gradient2d(img)
    assert np.array_equal(grad_d.cpu().numpy(), grad)
    levels, counts = oracle.segment(grad, 4, 3)
    assert c_d.cpu().tolist() == counts.tolist()
    assert np.array_equal(lv_d.cpu().numpy(), levels)


@pytest.fixture(scope="module")
def blob4096():
    img = synth.blob_image(4096, 4096, 2000, synth.BASE_SEED + 1)
    return img


@pytest.mark.parametrize("conn", [4, 8])
def test_blob_4096_quantised(ctx, blob4096, conn):
    img_d = torch.from_numpy(blob4096).cuda()
    grad_d = ctx.gradient(img_d, 4)
    lv_d, c_d = ctx.segment(grad_d, conn, 6)
    ctx.check()
    grad = oracle.gradient2d(blob4096, 4)
    assert np.array_equal(grad_d.cpu().numpy(), grad)
    levels, counts = oracle.segment(grad, conn, 6)
    assert c_d.cpu().tolist() == counts.tolist()
    got = lv_d.cpu().numpy()
    for k in range(6):
        assert np.array_equal(got[k], levels[k]), f"level {k}"


def _check_levels_properties(lv, counts):
    """Canonical ids, nesting and counts, on the device."""
    NL = lv.shape[0]
    N = lv[0].numel()
    ar = torch.arange(N, device=lv.device, dtype=torch.int64)
    prev = None
    for k in range(NL):
        L = lv[k].reshape(-1).long()
        K = counts[k]
        assert int(L.min()) == 0 and int(L.max()) == K - 1
        first = torch.full((K,), N, dtype=torch.int64, device=lv.device).scatter_reduce_(0, L, ar, "amin")
        assert bool((first[1:] > first[:-1]).all()), "not canonical"
        if prev is not None:
            m = torch.full((counts[k - 1],), -1, dtype=torch.int64, device=lv.device).scatter_(0, prev, L)
            assert bool((m[prev] == L).all()), "level not nested"
            assert counts[k] <= counts[k - 1]
        prev = L


@pytest.fixture(scope="module")
def vol928():
    return synth.distance_volume(928, 928, 928, 50000, seed=synth.BASE_SEED + 2)


def test_volume_928_properties(ctx, vol928):
    from scipy import ndimage
    grad_d = torch.from_numpy(vol928).cuda()
    lv_d, c_d = ctx.segment(grad_d, 6, 6)
    ctx.check()
    counts = c_d.cpu().tolist()
    _check_levels_properties(lv_d, counts)
    # minimal plateaux: components of {voxels with no strictly lower 6-neighbour}
    # (two adjacent such voxels are necessarily equal, so the components are
    # exactly the regional minima)
    g = grad_d.to(torch.int32)
    low = torch.zeros_like(g, dtype=torch.bool)
    for dim in range(3):
        n = g.shape[dim]
        a = g.narrow(dim, 1, n - 1)
        b = g.narrow(dim, 0, n - 1)
        low.narrow(dim, 1, n - 1).logical_or_(b < a)
        low.narrow(dim, 0, n - 1).logical_or_(a < b)
    mask = (~low).cpu().numpy()
    del g, low
    comp, ncomp = ndimage.label(mask, structure=ndimage.generate_binary_structure(3, 1))
    assert counts[0] == ncomp, f"K0 = {counts[0]} but {ncomp} regional minima"
    idx = np.flatnonzero(mask.ravel())
    cid = comp.ravel()[idx] - 1
    lab = lv_d[0].reshape(-1)[torch.from_numpy(idx).cuda()].cpu().numpy()
    lo = np.full(ncomp, np.iinfo(np.int64).max)
    hi = np.full(ncomp, -1)
    np.minimum.at(lo, cid, lab)
    np.maximum.at(hi, cid, lab)
    assert np.array_equal(lo, hi), "a minimal plateau split across basins"
    assert len(np.unique(lo)) == ncomp, "two minima in one basin"


def test_volume_928_vs_oracle(ctx, vol928):
    grad_d = torch.from_numpy(vol928).cuda()
    lv_d, c_d = ctx.segment(grad_d, 6, 6)
    ctx.check()
    levels, counts = oracle.segment(vol928, 6, 6)
    assert c_d.cpu().tolist() == counts.tolist()
    for k in range(6):
        assert torch.equal(lv_d[k].cpu(), torch.from_numpy(levels[k])), f"level {k}"


def _compare_many(items, got, what):
    """items: [(array, conn, NL)]; got: [(levels (CPU), counts list)], same order."""
    from oracle_pool import OraclePool, digest, first_difference
    with OraclePool() as pool:
        want = pool.segment_digests(items)
    bad = [i for i, ((lv, cnt), (wc, wd)) in enumerate(zip(got, want)) if cnt != wc or digest(lv) != wd]
    if bad:
        i = bad[0]
        arr, conn, NL = items[i]
        levels, counts = oracle.segment(arr, conn, NL)
        msg = [f"{what}: {len(bad)} of {len(items)} differ from the oracle; first: item {i}, shape {arr.shape}, "
               f"counts {got[i][1]} vs {counts.tolist()}"]
        for k in range(NL):
            msg.append(f"level {k}: " + first_difference(np.asarray(got[i][0][k]), levels[k]))
        pytest.fail("; ".join(msg))


def test_batch_512_vs_oracle(ctx):
    """The bench's 512-image batch, replayed from its CUDA graph: every image
    against the oracle (and the pool gradient too)."""
    img = synth.crop_pool_image(synth.BATCH_POOL_SEED)
    pool_d = ctx.gradient(torch.from_numpy(img).cuda())
    ctx.check()
    pool = oracle.gradient2d(img)
    assert np.array_equal(pool_d.cpu().numpy(), pool)
    wins = synth.batch_windows(512)
    grads = [pool_d[y:y + h, x:x + w].contiguous() for y, x, h, w in wins]
    g = ctx.graph(grads, 4, 6)
    ctx.check()
    for lv in g.levels:
        lv.fill_(-7)
    g.launch()
    ctx.check()
    got = [(lv.cpu().numpy(), c.cpu().tolist()) for lv, c in zip(g.levels, g.counts)]
    g.close()
    items = [(np.ascontiguousarray(pool[y:y + h, x:x + w]), 4, 6) for y, x, h, w in wins]
    _compare_many(items, got, "512-image batch")


def test_served_mix_vs_oracle(ctx):
    """The first 200 requests of the request stream (2D uint8 256..4096, 3D
    uint16 64..256, NL = 4) queued at once on a four-lane server with the
    bench's budget and batch limit, device-resident: every result against the
    oracle."""
    from paper_2410_08946_gb300 import binding
    NL = 4
    img = synth.crop_pool_image(synth.SERVE_SEED)
    pool2_d = ctx.gradient(torch.from_numpy(img).cuda())
    ctx.check()
    pool2 = oracle.gradient2d(img)
    assert np.array_equal(pool2_d.cpu().numpy(), pool2)
    vs = synth.SERVE_VOLUME_SIDE
    pool3 = synth.distance_volume(vs, vs, vs, synth.SERVE_VOLUME_SEEDS, seed=synth.SERVE_SEED)
    pool3_d = torch.from_numpy(pool3).cuda()
    reqs = synth.request_stream(200.0, 60.0, seed=synth.SERVE_SEED)[:200]
    assert 20 <= sum(r["kind"] == "3d" for r in reqs) <= 60
    items, dev = [], []
    for i, r in enumerate(reqs):
        if r["kind"] == "2d":
            h, w = r["shape"]
            y, x = synth.request_window_2d(i, h, w)
            items.append((np.ascontiguousarray(pool2[y:y + h, x:x + w]), 4, NL))
            dev.append(pool2_d[y:y + h, x:x + w].contiguous())
        else:
            d, h, w = r["shape"]
            items.append((np.ascontiguousarray(pool3[:d, :h, :w]), 6, NL))
            dev.append(pool3_d[:d, :h, :w].contiguous())
    got = []
    with binding.Server(0, budget_bytes=40 << 30, lanes=4, max_batch=64) as srv:
        tickets = [srv.submit(t, conn, NL) for t, (_, conn, _) in zip(dev, items)]
        for tk in tickets:
            st, lv, cnt = srv.poll(tk, 600_000_000)
            assert st == binding.WS_OK
            got.append((lv.cpu().numpy(), cnt.cpu().tolist()))
    _compare_many(items, got, "served mix")
