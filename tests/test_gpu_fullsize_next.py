"""The NEXT rows at full size, on the bench's volumes.

  region graph   of level planes 0 and 3 of the 928^3 6-connectivity
                 segmentation: CSR invariants, sizes and value sums against
                 torch.bincount, pass values of sampled edges recomputed from
                 every voxel pair of the two regions, and the graph-form
                 waterfall rule on the exported graph rebuilding the next level
  3D gradient    of the 928^3 volume: sampled blocks (interior and the eight
                 corners, where the replicated border acts) against the oracle
                 run on crops with a 3-voxel margin (the reach of blur + Sobel)
  literal waterfall  on a 192^3 volume, element by element against the oracle

The oracle cannot run the 928^3 cases whole in test time, so those are checked
by sampled outputs and by properties that hold at any size."""
import numpy as np
import pytest

import oracle
from paper_2410_08946_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIDE, SEEDS, NL = 928, 50000, 6
OFFS = [(0, 0, 1), (0, 1, 0), (1, 0, 0)]   # forward neighbours (dz, dy, dx) of 6-connectivity


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
def vol928():
    return synth.distance_volume(SIDE, SIDE, SIDE, SEEDS, seed=synth.BASE_SEED + 2)


@pytest.fixture(scope="module")
def seg928(ctx, vol928):
    v = torch.from_numpy(vol928).cuda()
    lv, c = ctx.segment(v, 6, NL)
    ctx.check()
    return v, lv, c.cpu().tolist()


def _brute_pass(L, G, A, B):
    """min over adjacent voxel pairs (one in A, one in B) of max(G(p), G(q))."""
    best = None
    for off in OFFS:
        dz, dy, dx = off
        D, H, W = L.shape
        l0, l1 = L[:D - dz, :H - dy, :W - dx], L[dz:, dy:, dx:]
        g0, g1 = G[:D - dz, :H - dy, :W - dx], G[dz:, dy:, dx:]
        m = ((l0 == A) & (l1 == B)) | ((l0 == B) & (l1 == A))
        if bool(m.any()):
            h = int(torch.maximum(g0[m], g1[m]).min())
            best = h if best is None else min(best, h)
    return best


def _components(K, rows, cols):
    """Connected components (min id labels) of an edge list, by min-label
    propagation on the GPU."""
    lab = torch.arange(K, device=rows.device)
    for _ in range(100000):
        new = lab.clone()
        new.scatter_reduce_(0, rows, lab[cols], reduce="amin")
        new.scatter_reduce_(0, cols, lab[rows], reduce="amin")
        new = new[new]   # jump
        if torch.equal(new, lab):
            return lab
        lab = new
    raise AssertionError("no convergence")


@pytest.mark.parametrize("level", [0, 3])
def test_region_graph_928(ctx, seg928, level):
    v, lv, counts = seg928
    L = lv[level]
    G = ctx.region_graph(L, v, 6, values=v)
    ctx.check()
    K = counts[level]
    N = L.numel()
    rp, col, pas = G["row_ptr"], G["col"].long(), G["pass"].long()
    assert rp.numel() == K + 1 and int(rp[0]) == 0 and int(rp[-1]) == col.numel()
    rows = torch.repeat_interleave(torch.arange(K, device=rp.device), torch.diff(rp))
    # no self-loops, columns strictly increasing within each row
    assert not bool((rows == col).any())
    key = rows * K + col
    assert bool((torch.diff(key) > 0).all())
    # symmetric with equal pass values
    rkey = col * K + rows
    order = torch.argsort(rkey)
    assert torch.equal(rkey[order], key) and torch.equal(pas[order], pas)
    # node features against bincount (independent of the library)
    Lf = L.reshape(-1).long()
    assert torch.equal(G["size"], torch.bincount(Lf, minlength=K))
    sums = torch.bincount(Lf, weights=v.reshape(-1).double(), minlength=K)   # exact: sums < 2^53
    assert torch.equal(G["sum"][:, 0].double(), sums)
    mean = torch.where(G["size"] > 0, G["sum"][:, 0].double() / G["size"].double(), torch.zeros_like(sums))
    assert torch.equal(G["mean"][:, 0], mean)
    # pass values of sampled edges, from every voxel pair of the two regions
    rng = np.random.default_rng(level)
    v32 = v.int()   # (uint16 CUDA tensors cannot be indexed by masks)
    for e in rng.choice(col.numel(), size=6, replace=False).tolist():
        A, B = int(rows[e]), int(col[e])
        assert _brute_pass(L, v32, A, B) == int(pas[e]), (A, B)
    del v32
    # the graph-form rule on the exported graph rebuilds the next level
    if level + 1 < NL:
        newmin = torch.full((K,), 1 << 40, dtype=torch.long, device=pas.device)
        newmin.scatter_reduce_(0, rows, pas, reduce="amin")
        keep = (pas == newmin[rows]) | (pas == newmin[col])
        comp = _components(K, rows[keep], col[keep])
        nxt = lv[level + 1].reshape(-1).long()
        first = torch.full((K,), N, dtype=torch.long, device=pas.device)
        first.scatter_reduce_(0, Lf, torch.arange(N, device=pas.device), reduce="amin")
        lab_next = nxt[first]                     # level k+1 id of each level-k region
        pairs = torch.unique(comp * (counts[level + 1] + 1) + lab_next)
        assert pairs.numel() == int(torch.unique(comp).numel()) == counts[level + 1]


def test_gradient3d_928_sampled(ctx, vol928):
    v = torch.from_numpy(vol928).cuda()
    g = ctx.gradient3d(v).cpu().numpy()
    ctx.check()
    S, R, B = SIDE, 3, 24
    rng = np.random.default_rng(7)
    starts = [tuple(int(t) for t in rng.integers(R, S - B - R, size=3)) for _ in range(6)]
    starts += [(z, y, x) for z in (0, S - B) for y in (0, S - B) for x in (0, S - B)]
    for z0, y0, x0 in starts:
        lo = [max(0, c - R) for c in (z0, y0, x0)]
        hi = [min(S, c + B + R) for c in (z0, y0, x0)]
        crop = np.ascontiguousarray(vol928[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])
        ref = oracle.gradient3d(crop)
        sl = tuple(slice(c - l, c - l + B) for c, l in zip((z0, y0, x0), lo))
        assert np.array_equal(g[z0:z0 + B, y0:y0 + B, x0:x0 + B], ref[sl]), (z0, y0, x0)


def test_waterfall_reconstruct_192(ctx):
    s = 192
    vol = synth.distance_volume(s, s, s, max(16, round(SEEDS * s ** 3 / SIDE ** 3)), seed=synth.BASE_SEED + 2)
    ref_l, ref_c = oracle.waterfall_reconstruct(vol, 6, 4)
    lv, c = ctx.waterfall_reconstruct(torch.from_numpy(vol).cuda(), 6, 4)
    ctx.check()
    assert c.cpu().tolist() == ref_c.tolist()
    assert np.array_equal(lv.cpu().numpy(), ref_l)
