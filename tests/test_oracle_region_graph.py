"""Pins of the oracle's region graph (Sec. 6: waterfall regions as the graph of
a graph network; edge weights are the pass values of Alg. 5 step V).

The region graph is defined by: an edge (A, B), A != B, exactly when a pixel of
A and a pixel of B are neighbours (Sec. 3.1, N(p)); its weight pass(A, B) is the
smallest max(G(p), G(q)) over those pixel pairs; node features are the pixel
count and per-channel sum and mean of a value image.  The pins below check the
oracle against an all-pairs scan that decides adjacency from coordinate
distances (not from a neighbour-offset table), closed forms on grids of
rectangular blocks, a hand-worked example, and the lowest-pass rule of the
graph-form waterfall, which must rebuild the (separately pinned) next level.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2410_08946_gb300 import synth


def brute_graph(L, g, conn, values=None):
    """All pairs of pixels; adjacency from the coordinate difference."""
    shape = L.shape
    coords = list(itertools.product(*[range(n) for n in shape]))
    K = int(L.max()) + 1
    passes = {}
    for p in coords:
        for q in coords:
            if p == q:
                continue
            d = [abs(a - b) for a, b in zip(p, q)]
            adj = sum(d) == 1 if conn in (4, 6) else max(d) == 1
            if not adj or L[p] == L[q]:
                continue
            key = (int(L[p]), int(L[q]))
            h = max(int(g[p]), int(g[q]))
            passes[key] = min(passes.get(key, h), h)
    row_ptr = np.zeros(K + 1, dtype=np.int64)
    col, pas = [], []
    for (a, b) in sorted(passes):
        row_ptr[a + 1] += 1
        col.append(b)
        pas.append(passes[(a, b)])
    row_ptr = np.cumsum(row_ptr)
    size = np.zeros(K, dtype=np.int64)
    C = 0 if values is None else values.shape[0]
    ssum = np.zeros((K, C), dtype=np.uint64)
    for p in coords:
        size[L[p]] += 1
        for c in range(C):
            ssum[L[p], c] += int(values[(c,) + p])
    return row_ptr, col, pas, size, ssum


def check_against(G, ref):
    row_ptr, col, pas, size, ssum = ref
    assert G["row_ptr"].tolist() == row_ptr.tolist()
    assert G["col"].tolist() == list(col)
    assert G["pass"].tolist() == list(pas)
    assert G["size"].tolist() == size.tolist()
    assert G["sum"].tolist() == ssum.tolist()


@pytest.mark.parametrize("shape,conn", [((4, 5), 4), ((4, 5), 8), ((5, 3), 8), ((3, 3, 4), 6),
                                        ((3, 3, 4), 26), ((2, 4, 3), 26)])
def test_brute_force_all_pairs(shape, conn):
    rng = np.random.default_rng(sum(shape) * conn)
    for trial in range(12):
        nlab = [1, 2, 3, 6][trial % 4]
        L = rng.integers(0, nlab, size=shape).astype(np.int32)
        dt = np.uint8 if trial % 2 else np.uint16
        g = rng.integers(0, 40 if dt == np.uint8 else 3000, size=shape).astype(dt)
        vals = rng.integers(0, 65535, size=(2,) + shape).astype(np.uint16)
        G = oracle.region_graph(L, g, conn, values=vals)
        check_against(G, brute_graph(L, g, conn, vals))
        K = int(L.max()) + 1
        with np.errstate(invalid="ignore", divide="ignore"):
            want = np.where(G["size"][:, None] > 0, G["sum"] / np.maximum(G["size"][:, None], 1), 0.0)
        assert np.array_equal(G["mean"], want)
        assert len(G["row_ptr"]) == K + 1


def test_hand_worked_example():
    """Labels     Gradient   (4-connectivity)
       0 0 1      1 2 3
       0 2 1      4 5 6
    Region pairs across a pixel edge: (0,1) at G 2|3 -> 3; (0,2) at 4|5 -> 5 and
    2|5 -> 5; (2,1) at 5|6 -> 6.  Sizes 3, 2, 1; sums of the gradient 7, 9, 5."""
    L = np.array([[0, 0, 1], [0, 2, 1]], dtype=np.int32)
    g = np.array([[1, 2, 3], [4, 5, 6]], dtype=np.uint8)
    G = oracle.region_graph(L, g, 4, values=g)
    assert G["row_ptr"].tolist() == [0, 2, 4, 6]
    assert G["col"].tolist() == [1, 2, 0, 2, 0, 1]
    assert G["pass"].tolist() == [3, 5, 3, 6, 5, 6]
    assert G["size"].tolist() == [3, 2, 1]
    assert G["sum"][:, 0].tolist() == [7, 9, 5]
    assert G["mean"][:, 0].tolist() == [7 / 3, 4.5, 5.0]
    # 8-connectivity adds the diagonal 0(0,1)-1(1,2) at max(2, 6) = 6 (not
    # lower than 3) and 2(1,1)-1(0,2) at max(5, 3) = 5, which lowers pass(1,2)
    G8 = oracle.region_graph(L, g, 8)
    assert G8["col"].tolist() == [1, 2, 0, 2, 0, 1]
    assert G8["pass"].tolist() == [3, 5, 3, 5, 5, 5]


@pytest.mark.parametrize("conn", [4, 8])
def test_block_grid_closed_form(conn):
    """R x C blocks of bh x bw pixels, block (r, c) labelled r*C + c, gradient
    G(x, y) = x + 10 y.  Horizontal neighbours meet on the column pair
    x0 - 1 | x0 (x0 = (c+1) bw): pass = x0 + 10 r bh; vertical ones on the row
    pair y0 - 1 | y0: pass = c bw + 10 y0.  With 8-connectivity the diagonal
    block pairs touch at one corner: (r,c)-(r+1,c+1) at max(G(x0-1, y0-1),
    G(x0, y0)) = x0 + 10 y0 and (r,c+1)-(r+1,c) at max(G(x0, y0-1),
    G(x0-1, y0)) = x0 - 1 + 10 y0; the extra diagonal pixel pairs of side
    neighbours are never lower than the straight ones."""
    R, C, bh, bw = 3, 4, 3, 5
    H, W = R * bh, C * bw
    y, x = np.mgrid[0:H, 0:W]
    g = (x + 10 * y).astype(np.uint16)
    L = ((y // bh) * C + (x // bw)).astype(np.int32)
    want = {}
    for r in range(R):
        for c in range(C):
            a = r * C + c
            if c + 1 < C:
                want[(a, a + 1)] = (c + 1) * bw + 10 * r * bh
            if r + 1 < R:
                want[(a, a + C)] = c * bw + 10 * (r + 1) * bh
            if conn == 8 and r + 1 < R and c + 1 < C:
                x0, y0 = (c + 1) * bw, (r + 1) * bh
                want[(a, a + C + 1)] = x0 + 10 * y0
                want[(a + 1, a + C)] = x0 - 1 + 10 * y0
    both = {}
    for (a, b), h in want.items():
        both[(a, b)] = h
        both[(b, a)] = h
    G = oracle.region_graph(L, g, conn, values=g)
    got = {}
    for a in range(R * C):
        for i in range(G["row_ptr"][a], G["row_ptr"][a + 1]):
            got[(a, int(G["col"][i]))] = int(G["pass"][i])
    assert got == both
    assert G["size"].tolist() == [bh * bw] * (R * C)
    for r in range(R):
        for c in range(C):
            xs = np.arange(c * bw, (c + 1) * bw)
            ys = np.arange(r * bh, (r + 1) * bh)
            assert int(G["sum"][r * C + c, 0]) == bh * xs.sum() + 10 * bw * ys.sum()
    # edge count of the grid graph (4) or the king's graph (8)
    E = R * (C - 1) + (R - 1) * C + (2 * (R - 1) * (C - 1) if conn == 8 else 0)
    assert len(G["col"]) == 2 * E


@pytest.mark.parametrize("conn", [6, 26])
def test_block_grid_3d_adjacency(conn):
    """3D blocks: with 6-connectivity block pairs one step apart along one axis
    are adjacent; with 26-connectivity every pair at Chebyshev distance 1 in
    block coordinates.  A constant gradient makes every pass that constant."""
    nb = (2, 3, 3)
    bs = (2, 3, 2)
    shape = tuple(n * s for n, s in zip(nb, bs))
    z, y, x = np.indices(shape)
    L = (((z // bs[0]) * nb[1] + (y // bs[1])) * nb[2] + (x // bs[2])).astype(np.int32)
    g = np.full(shape, 7, dtype=np.uint8)
    G = oracle.region_graph(L, g, conn)
    blocks = list(itertools.product(*[range(n) for n in nb]))
    idx = {b: (b[0] * nb[1] + b[1]) * nb[2] + b[2] for b in blocks}
    for b in blocks:
        d = [[abs(u - v) for u, v in zip(b, o)] for o in blocks]
        nbrs = sorted(idx[o] for o, dd in zip(blocks, d) if o != b and
                      (sum(dd) == 1 if conn == 6 else max(dd) == 1))
        a = idx[b]
        assert G["col"][G["row_ptr"][a]:G["row_ptr"][a + 1]].tolist() == nbrs
    assert set(G["pass"].tolist()) == {7}


def _components(K, edges):
    par = list(range(K))

    def find(a):
        while par[a] != a:
            par[a] = par[par[a]]
            a = par[a]
        return a
    for a, b in edges:
        ra, rb = find(a), find(b)
        if ra != rb:
            par[max(ra, rb)] = min(ra, rb)
    return [find(a) for a in range(K)]


@pytest.mark.parametrize("shape,conn", [((40, 50), 4), ((40, 50), 8), ((12, 14, 16), 6), ((10, 12, 9), 26)])
def test_lowest_pass_rule_rebuilds_next_level(shape, conn):
    """Graph-form waterfall (Alg. 5 steps V-VI on the region graph): keeping the
    edges whose pass is the lowest pass of one endpoint and taking connected
    components of level k must give exactly the partition of level k + 1."""
    v = synth.distance_volume(1, *shape, 25, seed=3)[0] if len(shape) == 2 else \
        synth.distance_volume(*shape, 25, seed=3)
    levels, counts = oracle.segment(v, conn, 4)
    for k in range(3):
        G = oracle.region_graph(levels[k], v, conn)
        K = int(counts[k])
        rows = np.repeat(np.arange(K), np.diff(G["row_ptr"]))
        newmin = np.full(K, np.iinfo(np.uint32).max, dtype=np.uint64)
        np.minimum.at(newmin, rows, G["pass"].astype(np.uint64))
        keep = (G["pass"] == newmin[rows]) | (G["pass"] == newmin[G["col"]])
        comp = np.array(_components(K, zip(rows[keep].tolist(), G["col"][keep].tolist())))
        nxt = levels[k + 1].ravel()
        cur = levels[k].ravel()
        # level k+1 is a function of the component, and distinct components differ
        pairs = set(zip(comp[cur].tolist(), nxt.tolist()))
        assert len(pairs) == len(set(comp.tolist())) == int(counts[k + 1])
        assert len({a for a, _ in pairs}) == len({b for _, b in pairs}) == len(pairs)


def test_invariants_random_segmentation():
    v = synth.distance_volume(1, 96, 80, 60, seed=9)[0]
    levels, counts = oracle.segment(v, 8, 3)
    vals = np.stack([v, (v >> 3).astype(np.uint16)])
    for k in range(3):
        G = oracle.region_graph(levels[k], v, 8, values=vals)
        K = int(counts[k])
        rp, col, pas = G["row_ptr"], G["col"], G["pass"]
        assert rp[0] == 0 and rp[-1] == len(col) and np.all(np.diff(rp) >= 0)
        d = {}
        for a in range(K):
            row = col[rp[a]:rp[a + 1]]
            assert np.all(np.diff(row) > 0) and a not in row.tolist()
            for i in range(rp[a], rp[a + 1]):
                d[(a, int(col[i]))] = int(pas[i])
        assert all(d[(b, a)] == h for (a, b), h in d.items())
        assert G["size"].sum() == v.size and np.all(G["size"] > 0)
        assert G["sum"].sum(axis=0).tolist() == [int(vals[0].sum()), int(vals[1].sum())]
        if k > 0:  # every region of a waterfall level above 0 has a neighbour unless it is alone
            assert K == 1 or np.all(np.diff(rp) > 0)


def test_single_region_and_gaps():
    g = np.arange(12, dtype=np.uint8).reshape(3, 4)
    G = oracle.region_graph(np.zeros((3, 4), np.int32), g, 4, values=g)
    assert G["row_ptr"].tolist() == [0, 0] and len(G["col"]) == 0
    assert G["size"].tolist() == [12] and G["sum"][0, 0] == 66
    L = np.zeros((3, 4), np.int32)
    L[:, 2:] = 3   # ids 1 and 2 carry no pixel
    G = oracle.region_graph(L, g, 4, values=g)
    assert G["row_ptr"].tolist() == [0, 1, 1, 1, 2]
    assert G["col"].tolist() == [3, 0] and G["pass"].tolist() == [2, 2]
    assert G["size"].tolist() == [6, 0, 0, 6] and G["mean"][1:3, 0].tolist() == [0.0, 0.0]
    with pytest.raises(ValueError):
        oracle.region_graph(L - 1, g, 4)
