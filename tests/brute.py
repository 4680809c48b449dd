"""Independent brute-force checkers used to pin the oracle (tiny inputs only).

Nothing here is imported by the product.  These are deliberately written in a
different style from the C oracle: the oracle computes the defined result
(BFS, root chasing), while this module *simulates the paper's iterations*
(Alg. 1 steps I-IV with the synchronous S/S' double buffer and the RR-bounded
path reduction, Alg. 3's block-asynchronous balanced resolution) or uses
all-pairs shortest paths (Floyd-Warshall) and exhaustive pair scans.  A
mistake in either style shows up as a disagreement.
"""
from __future__ import annotations

import itertools
from collections import deque

import numpy as np


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def offsets(ndim: int, conn: int):
    offs = []
    for d in itertools.product((-1, 0, 1), repeat=3):
        dz, dy, dx = d
        if d == (0, 0, 0):
            continue
        if ndim == 2 and dz != 0:
            continue
        l1 = abs(dx) + abs(dy) + abs(dz)
        if conn in (4, 6) and l1 != 1:
            continue
        offs.append((dz, dy, dx))
    return offs


class Grid:
    """Flat indexing over an image of shape (H, W) or (D, H, W)."""

    def __init__(self, shape, conn):
        if len(shape) == 1:
            shape = (1, shape[0])
        self.ndim = len(shape)
        self.shape3 = (1,) * (3 - self.ndim) + tuple(shape)
        self.D, self.H, self.W = self.shape3
        self.N = self.D * self.H * self.W
        self.conn = conn
        self.offs = offsets(self.ndim, conn)
        self._nb = []
        for p in range(self.N):
            z, r = divmod(p, self.H * self.W)
            y, x = divmod(r, self.W)
            lst = []
            for dz, dy, dx in self.offs:
                zz, yy, xx = z + dz, y + dy, x + dx
                if 0 <= zz < self.D and 0 <= yy < self.H and 0 <= xx < self.W:
                    lst.append((zz * self.H + yy) * self.W + xx)
            self._nb.append(lst)

    def nb(self, p):
        return self._nb[p]


def canonical(labels: np.ndarray) -> np.ndarray:
    """Relabel to 0..K-1 in order of first appearance (smallest pixel index)."""
    flat = np.asarray(labels).ravel()
    out = np.empty(flat.shape, dtype=np.int64)
    seen = {}
    for i, v in enumerate(flat.tolist()):
        if v not in seen:
            seen[v] = len(seen)
        out[i] = seen[v]
    return out.reshape(np.asarray(labels).shape)


# --------------------------------------------------------------------------
# literal simulation of Alg. 1 (PRUF, synchronous step II)
# --------------------------------------------------------------------------

def literal_step1(I, G: Grid):
    """Eq. 1 literally: q = max{ r in N(p) : I(r) <= I(n) for all n in N(p) }."""
    S = [0] * G.N
    L = [0] * G.N
    for p in range(G.N):
        nbs = G.nb(p)
        if not nbs:
            S[p], L[p] = 1, p
            continue
        cand = [r for r in nbs if all(I[r] <= I[n] for n in nbs)]
        q = max(cand)
        if I[q] < I[p]:
            S[p], L[p] = 0, q
        elif I[q] > I[p]:
            S[p], L[p] = 1, p
        elif q > p:
            S[p], L[p] = 2, q
        else:
            S[p], L[p] = 3, p
    return S, L


def literal_alg1(grad: np.ndarray, conn: int, RR: int = 6, return_trace: bool = False):
    """Alg. 1 run literally on a tiny image.

    Step II: synchronous rounds with the S' buffer; a plateau pixel that sees
    an equal-valued state-0 neighbour in the *previous* round's S takes it as
    its label.  When several qualify, the largest index is taken (the reading
    the oracle states; the paper only says "there exists").
    Step III: rounds of at most RR jumps per pixel, each round reading the
    labels as they were at its start; repeat until no label changes.
    Step IV: Union over state>=2 neighbours with q > p, then Find.
    """
    I = [int(v) for v in np.asarray(grad).ravel().tolist()]
    G = Grid(np.asarray(grad).shape, conn)
    S, L = literal_step1(I, G)
    S1 = list(S)
    it2 = 0
    while True:
        it2 += 1
        Sn = list(S)
        Ln = list(L)
        change = False
        for p in range(G.N):
            if S[p] >= 2:
                cand = [q for q in G.nb(p) if S[q] == 0 and I[q] == I[p]]
                if cand:
                    Ln[p] = max(cand)
                    Sn[p] = 0
                    change = True
        S, L = Sn, Ln
        if not change:
            break
    L2 = list(L)
    it3 = 0
    while True:
        it3 += 1
        old = list(L)
        change = False
        for p in range(G.N):
            lab = old[p]
            for _ in range(RR):
                if lab == old[lab]:
                    break
                lab = old[lab]
            if lab != L[p]:
                L[p] = lab
                change = True
        if not change:
            break
    # step IV: sequential Union-Find on the label array itself
    par = list(L)

    def find(a):
        while par[a] != a:
            a = par[a]
        return a

    for p in range(G.N):
        if S[p] >= 2:
            for q in G.nb(p):
                if q > p and S[q] >= 2:
                    ra, rb = find(p), find(q)
                    if ra != rb:
                        par[max(ra, rb)] = min(ra, rb)
    final = [find(p) for p in range(G.N)]
    out = np.array(final, dtype=np.int64).reshape(np.asarray(grad).shape)
    if return_trace:
        return out, dict(S1=S1, L2=L2, it2=it2, it3=it3, S2=S)
    return out


def step3_rounds(L, RR):
    """Number of RR-bounded path-reduction rounds (Alg. 1 step III) until the
    labels stop changing, counting the final round that changes nothing."""
    L = list(L)
    rounds = 0
    while True:
        rounds += 1
        old = list(L)
        change = False
        for p in range(len(L)):
            lab = old[p]
            for _ in range(RR):
                if lab == old[lab]:
                    break
                lab = old[lab]
            if lab != L[p]:
                L[p] = lab
                change = True
        if not change:
            return rounds, L


# --------------------------------------------------------------------------
# literal simulation of Alg. 3 (PRUF_bal), 1D blocks
# --------------------------------------------------------------------------

def literal_bal_1d(values, block: int):
    """Alg. 3 on a 1D image with 2-connectivity and blocks of `block` pixels.
    Returns the list of state vectors after every global iteration (until a
    global iteration changes nothing; that last one is not returned)."""
    I = list(values)
    n = len(I)
    G = Grid((n,), 4)
    S, _ = literal_step1(I, G)
    history = []
    while True:
        Sg = list(S)          # global memory at the start of this iteration
        Snew = list(S)
        for b0 in range(0, n, block):
            idx = list(range(b0, min(n, b0 + block)))
            loc = {p: Sg[p] for p in idx}   # shared memory; halo frozen at Sg
            while True:
                changed = False
                snap = dict(loc)           # read phase (between SyncThreads)

                def st_snap(q):
                    return snap[q] if q in snap else Sg[q]

                for p in idx:
                    sp = snap[p]
                    best = None
                    for q in G.nb(p):
                        if I[q] != I[p]:
                            continue
                        sq = st_snap(q)
                        if (sp >= 2 and sq <= 0) or (sp + 1 < sq <= 0):
                            cand = sq - 1
                            if best is None or cand > best:
                                best = cand
                    if best is not None and (sp >= 2 or best > sp):
                        loc[p] = best
                        changed = True
                if not changed:
                    break
            for p in idx:
                Snew[p] = loc[p]
        if Snew == S:
            break
        S = Snew
        history.append(list(S))
    return history


# --------------------------------------------------------------------------
# Floyd-Warshall plateau distances
# --------------------------------------------------------------------------

def floyd_warshall_distance(grad: np.ndarray, conn: int, S):
    """d(p) = shortest equal-valued path from p to any state-0 pixel of its
    plateau, via all-pairs shortest paths; 0 for state 0, -1 when unreachable
    or state 1."""
    I = [int(v) for v in np.asarray(grad).ravel().tolist()]
    G = Grid(np.asarray(grad).shape, conn)
    INF = 10 ** 9
    n = G.N
    D = np.full((n, n), INF, dtype=np.int64)
    for p in range(n):
        D[p, p] = 0
        for q in G.nb(p):
            if I[q] == I[p]:
                D[p, q] = 1
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    S = list(np.asarray(S).ravel().tolist())
    out = []
    zero = [q for q in range(n) if S[q] == 0]
    for p in range(n):
        if S[p] == 0:
            out.append(0)
        elif S[p] == 1:
            out.append(-1)
        else:
            best = min((D[p, q] for q in zero), default=INF)
            out.append(int(best) if best < INF else -1)
    return np.array(out, dtype=np.int64).reshape(np.asarray(grad).shape)


# --------------------------------------------------------------------------
# waterfall by exhaustive pair scan
# --------------------------------------------------------------------------

def brute_waterfall(labels0: np.ndarray, grad: np.ndarray, conn: int, NL: int):
    I = [int(v) for v in np.asarray(grad).ravel().tolist()]
    G = Grid(np.asarray(grad).shape, conn)
    cur = [int(v) for v in np.asarray(labels0).ravel().tolist()]
    levels = [np.array(cur).reshape(np.asarray(grad).shape)]
    for _ in range(1, NL):
        passes = {}
        for p in range(G.N):
            for q in G.nb(p):
                a, b = cur[p], cur[q]
                if a == b:
                    continue
                key = (min(a, b), max(a, b))
                h = max(I[p], I[q])
                passes[key] = min(passes.get(key, h), h)
        newmin = {}
        for (a, b), h in passes.items():
            newmin[a] = min(newmin.get(a, h), h)
            newmin[b] = min(newmin.get(b, h), h)
        adj = {}
        for (a, b), h in passes.items():
            if h == newmin[a] or h == newmin[b]:
                adj.setdefault(a, []).append(b)
                adj.setdefault(b, []).append(a)
        comp = {}
        for r in sorted(set(cur)):
            if r in comp:
                continue
            comp[r] = r
            dq = deque([r])
            while dq:
                u = dq.popleft()
                for v in adj.get(u, []):
                    if v not in comp:
                        comp[v] = r
                        dq.append(v)
        nxt = [comp[c] for c in cur]
        cur = canonical(np.array(nxt)).ravel().tolist()
        levels.append(np.array(cur).reshape(np.asarray(grad).shape))
    return levels


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def regional_minima(grad: np.ndarray, conn: int):
    """Independent CCL: list of minimal plateaux (sets of pixels), found as
    equal-valued components with no strictly lower neighbour."""
    I = [int(v) for v in np.asarray(grad).ravel().tolist()]
    G = Grid(np.asarray(grad).shape, conn)
    seen = [False] * G.N
    out = []
    for s in range(G.N):
        if seen[s]:
            continue
        comp = []
        dq = deque([s])
        seen[s] = True
        while dq:
            u = dq.popleft()
            comp.append(u)
            for v in G.nb(u):
                if not seen[v] and I[v] == I[s]:
                    seen[v] = True
                    dq.append(v)
        lower = any(I[v] < I[s] for u in comp for v in G.nb(u))
        if not lower:
            out.append(comp)
    return out


def check_watershed_invariants(labels: np.ndarray, grad: np.ndarray, conn: int):
    lab = np.asarray(labels).ravel().tolist()
    G = Grid(np.asarray(grad).shape, conn)
    K = max(lab) + 1
    assert sorted(set(lab)) == list(range(K)), "labels not 0..K-1"
    # canonical order: region i first appears before region i+1
    first = {}
    for p, v in enumerate(lab):
        first.setdefault(v, p)
    assert all(first[i] < first[i + 1] for i in range(K - 1)), "not canonical"
    # each region connected
    members = {}
    for p, v in enumerate(lab):
        members.setdefault(v, []).append(p)
    for v, ps in members.items():
        s = set(ps)
        seen = {ps[0]}
        dq = deque([ps[0]])
        while dq:
            u = dq.popleft()
            for w in G.nb(u):
                if w in s and w not in seen:
                    seen.add(w)
                    dq.append(w)
        assert len(seen) == len(ps), f"region {v} not connected"
    # one regional minimum per region, K = number of minima
    mins = regional_minima(grad, conn)
    assert len(mins) == K, f"K={K} but {len(mins)} regional minima"
    hit = {}
    for comp in mins:
        ids = {lab[p] for p in comp}
        assert len(ids) == 1, "a minimal plateau split across regions"
        (i,) = ids
        assert i not in hit, "two minima in one region"
        hit[i] = True


def check_nested(levels):
    """Each level a union of regions of the level below; counts non-increasing."""
    counts = []
    for k, L in enumerate(levels):
        flat = np.asarray(L).ravel()
        counts.append(int(flat.max()) + 1)
        if k == 0:
            continue
        prev = np.asarray(levels[k - 1]).ravel()
        m = {}
        for a, b in zip(prev.tolist(), flat.tolist()):
            assert m.setdefault(a, b) == b, "level not nested"
    assert all(counts[i] >= counts[i + 1] for i in range(len(counts) - 1)), counts
    return counts
