"""Pins of the oracle's paper-literal waterfall: Alg. 4 with the image
reconstruction of Alg. 5 (step V: newmin of every region = its lowest
max(I(p), I(q)) across its border; step VI: raise the region's pixels below
newmin to it; then the watershed of the raised image).

The pins: a hand-derived 1D example (where the literal form is not nested
while the graph form is), and a replay of steps V-VI in Python that decides
adjacency from coordinate distances and calls the separately pinned oracle
watershed between levels."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2410_08946_gb300 import synth


def test_hand_derived_1d():
    """I = [10, 100, 50, 200, 80, 90, 5] (a 1x7 image, 4-connectivity).
    Level 0 (Eq. 1): 10 <- 100, 50 <- 200, 80 is a minimum, 5 <- 90:
    {0,1} {2,3} {4} {5,6}.  Step V: newmin = 100 (100|50), 100 (50|100 and
    200|80 -> 200), 90 (80|90), 90 (90|80).  Step VI: [100,100,100,200,90,90,90].
    Level 1: {0,1,2} is a minimal plateau at 100; 200 drains to the lower of
    100 and 90, i.e. to {4,5,6}: {0,1,2} {3,4,5,6}, so pixel 3 leaves its
    level-0 basin {2,3}.  Step V: both regions meet at 100|200 -> 200; step VI
    makes the image flat: level 2 is one region.  The graph form puts pixel 3
    with {0,1,2} instead (every level a union of level-0 basins)."""
    g = np.array([[10, 100, 50, 200, 80, 90, 5]], dtype=np.uint8)
    levels, counts = oracle.waterfall_reconstruct(g, 4, 3)
    assert counts.tolist() == [4, 2, 1]
    assert levels[0, 0].tolist() == [0, 0, 1, 1, 2, 3, 3]
    assert levels[1, 0].tolist() == [0, 0, 0, 1, 1, 1, 1]
    assert levels[2, 0].tolist() == [0] * 7
    glev, gcnt = oracle.segment(g, 4, 3)
    assert gcnt.tolist() == [4, 2, 1]
    assert glev[1, 0].tolist() == [0, 0, 0, 0, 1, 1, 1]


def replay(g, conn, NL):
    """Alg. 4 / Alg. 5 literally, with the pinned oracle watershed per level."""
    shape = g.shape
    coords = list(itertools.product(*[range(n) for n in shape]))
    M = np.iinfo(g.dtype).max
    I = g.copy()
    out = []
    for n in range(NL):
        L, K = oracle.watershed(I, conn)
        out.append(L)
        if n == NL - 1:
            break
        newmin = [M] * K
        for p in coords:
            for q in coords:
                d = [abs(a - b) for a, b in zip(p, q)]
                adj = sum(d) == 1 if conn in (4, 6) else max(d) == 1
                if adj and L[p] != L[q]:
                    newmin[L[p]] = min(newmin[L[p]], max(int(I[p]), int(I[q])))
        I = I.copy()
        for p in coords:
            if I[p] < newmin[L[p]]:
                I[p] = newmin[L[p]]
    return np.stack(out)


@pytest.mark.parametrize("shape,conn", [((5, 6), 4), ((5, 6), 8), ((4, 7), 8), ((3, 3, 4), 6), ((3, 3, 3), 26)])
def test_replay_steps_v_vi(shape, conn):
    rng = np.random.default_rng(sum(shape) + conn)
    for trial in range(6):
        dt = np.uint8 if trial % 2 == 0 else np.uint16
        hi = [4, 10, 300][trial % 3]
        g = rng.integers(0, min(hi, np.iinfo(dt).max), size=shape).astype(dt)
        levels, counts = oracle.waterfall_reconstruct(g, conn, 4)
        ref = replay(g, conn, 4)
        assert np.array_equal(levels, ref), (g.tolist(), conn)
        assert counts.tolist() == [int(l.max()) + 1 for l in ref]


def test_flat_and_single_region():
    for dt in (np.uint8, np.uint16):
        g = np.full((6, 9), 7, dtype=dt)
        levels, counts = oracle.waterfall_reconstruct(g, 8, 3)
        assert counts.tolist() == [1, 1, 1] and not levels.any()
    g = np.array([[3, 2, 1, 2, 3]], dtype=np.uint8)   # one basin: stays one region
    levels, counts = oracle.waterfall_reconstruct(g, 4, 4)
    assert counts.tolist() == [1, 1, 1, 1]


def test_level0_is_the_watershed():
    """Level 0 is the watershed of the input in both forms (above it the
    literal form may leave the graph form's nesting, as in the 1D example)."""
    for conn, shape in [(4, (1, 64, 80)), (8, (1, 96, 96)), (6, (16, 20, 24)), (26, (12, 14, 16))]:
        v = synth.distance_volume(*shape, 60, seed=5)
        if shape[0] == 1:
            v = v[0]
        lit, lc = oracle.waterfall_reconstruct(v, conn, 3)
        gra, gc = oracle.segment(v, conn, 3)
        assert np.array_equal(lit[0], gra[0]) and lc[0] == gc[0]
        assert np.array_equal(lit[0], oracle.watershed(v, conn)[0])
