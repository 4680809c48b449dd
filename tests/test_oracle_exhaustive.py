"""Exhaustive and randomised tiny-image pins of the oracle against the
literal simulation of Alg. 1 (tests/brute.py), Floyd-Warshall plateau
distances, a brute-force waterfall and the watershed invariants."""
import itertools

import numpy as np
import pytest

import oracle
from brute import (Grid, canonical, literal_alg1, literal_step1, floyd_warshall_distance,
                   brute_waterfall, check_watershed_invariants, check_nested)


def _all_images(shape, levels):
    n = int(np.prod(shape))
    for vals in itertools.product(range(levels), repeat=n):
        yield np.array(vals, dtype=np.uint8).reshape(shape)


def _check_one(img, conn, full=False):
    labels, K, S1, dist, ptr = oracle.watershed(img, conn, debug=True)
    ref, tr = literal_alg1(img, conn, return_trace=True)
    assert np.array_equal(canonical(ref), labels), (img.tolist(), conn)
    assert S1.ravel().tolist() == tr["S1"]
    assert ptr.ravel().tolist() == tr["L2"]
    assert K == labels.max() + 1
    if full:
        fw = floyd_warshall_distance(img, conn, S1)
        assert np.array_equal(fw, dist), (img.tolist(), conn)
        check_watershed_invariants(labels, img, conn)


@pytest.mark.parametrize("conn", [4, 8])
def test_exhaustive_3x3(conn):
    for i, img in enumerate(_all_images((3, 3), 3)):
        _check_one(img, conn, full=(i % 97 == 0))


@pytest.mark.parametrize("shape", [(2, 4), (4, 2)])
@pytest.mark.parametrize("conn", [4, 8])
def test_exhaustive_2x4(shape, conn):
    for i, img in enumerate(_all_images(shape, 3)):
        _check_one(img, conn, full=(i % 53 == 0))


def test_exhaustive_1d():
    for n in range(1, 7):
        for img in _all_images((1, n), 4):
            _check_one(img, 4, full=True)


@pytest.mark.parametrize("conn", [6, 26])
def test_exhaustive_2x2x2(conn):
    for i, img in enumerate(_all_images((2, 2, 2), 3)):
        _check_one(img, conn, full=(i % 41 == 0))


@pytest.mark.parametrize("seed", range(30))
@pytest.mark.parametrize("conn", [4, 8])
def test_random_2d(seed, conn):
    rng = np.random.default_rng(1000 + seed)
    H, W = rng.integers(1, 13, size=2)
    levels = int(rng.integers(2, 6))
    img = rng.integers(0, levels, size=(H, W)).astype(np.uint8)
    _check_one(img, conn, full=True)


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("conn", [6, 26])
def test_random_3d(seed, conn):
    rng = np.random.default_rng(2000 + seed)
    D, H, W = rng.integers(1, 6, size=3)
    levels = int(rng.integers(2, 5))
    img = rng.integers(0, levels, size=(D, H, W)).astype(np.uint16) * 1000
    _check_one(img, conn, full=True)


def test_step1_uint16_matches_literal():
    rng = np.random.default_rng(7)
    img = rng.integers(0, 65536, size=(9, 11)).astype(np.uint16)
    img[2:5, 3:7] = 40000          # a plateau
    for conn in (4, 8):
        S, L = oracle.step1(img, conn)
        G = Grid(img.shape, conn)
        S2, L2 = literal_step1([int(v) for v in img.ravel()], G)
        assert S.ravel().tolist() == S2 and L.ravel().tolist() == L2


# --------------------------------------------------------------------------
# special cases
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,conn", [((1, 1), 4), ((1, 1, 1), 6), ((7, 5), 4), ((7, 5), 8),
                                         ((3, 4, 5), 6), ((3, 4, 5), 26)])
def test_constant_image_one_region(shape, conn):
    for v in (0, 255):
        img = np.full(shape, v, dtype=np.uint8)
        labels, K = oracle.watershed(img, conn)
        assert K == 1 and not labels.any()


@pytest.mark.parametrize("conn", [4, 8])
def test_monotone_ramp_one_region(conn):
    y, x = np.mgrid[0:9, 0:13]
    img = (x + 2 * y).astype(np.uint8)
    labels, K = oracle.watershed(img, conn)
    assert K == 1


def test_checkerboard_one_region_per_low_pixel():
    y, x = np.mgrid[0:8, 0:10]
    img = ((x + y) % 2).astype(np.uint8) * 9
    labels, K = oracle.watershed(img, 4)
    assert K == int((img == 0).sum())
    check_watershed_invariants(labels, img, 4)


def test_max_value_plateau_uint16():
    img = np.full((6, 6), 65535, dtype=np.uint16)
    img[0, 0] = 65534
    labels, K = oracle.watershed(img, 4)
    assert K == 1
    img[5, 5] = 65534
    labels, K = oracle.watershed(img, 4)
    assert K == 2
    # the flat plateau splits by distance: pixel (r, c) joins the nearer corner
    lab = labels.tolist()
    for r in range(6):
        for c in range(6):
            d0, d1 = r + c, (5 - r) + (5 - c)
            if d0 < d1:
                assert lab[r][c] == 0
            elif d1 < d0:
                assert lab[r][c] == 1


# --------------------------------------------------------------------------
# waterfall
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(40))
@pytest.mark.parametrize("conn", [4, 8])
def test_waterfall_vs_bruteforce(seed, conn):
    rng = np.random.default_rng(3000 + seed)
    H, W = rng.integers(2, 12, size=2)
    img = rng.integers(0, 6, size=(H, W)).astype(np.uint8)
    L0, K = oracle.watershed(img, conn)
    NL = 5
    levels, counts = oracle.waterfall(L0, img, conn, NL)
    ref = brute_waterfall(L0, img, conn, NL)
    for k in range(1, NL):
        assert np.array_equal(levels[k - 1], ref[k]), k
    got = check_nested([L0] + list(levels))
    assert got == counts.tolist()


@pytest.mark.parametrize("seed", range(10))
def test_waterfall_3d_vs_bruteforce(seed):
    rng = np.random.default_rng(4000 + seed)
    D, H, W = rng.integers(2, 6, size=3)
    img = rng.integers(0, 5, size=(D, H, W)).astype(np.uint16)
    L0, K = oracle.watershed(img, 6)
    levels, counts = oracle.waterfall(L0, img, 6, 4)
    ref = brute_waterfall(L0, img, 6, 4)
    for k in range(1, 4):
        assert np.array_equal(levels[k - 1], ref[k])


def test_waterfall_two_basins_merge():
    img = np.array([[1, 5, 9, 5, 0]], dtype=np.uint8)
    L0, K = oracle.watershed(img, 4)
    assert K == 2
    levels, counts = oracle.waterfall(L0, img, 4, 3)
    assert counts.tolist() == [2, 1, 1]
    assert not levels.any()


def test_waterfall_graph_form_counterexample():
    """The 1D image where re-running the pixel watershed on the reconstructed
    image (Alg. 5 + Alg. 4) is not nested; the graph form keeps level 0's
    basins whole.  Level 0: {0,1} {2,3} {4} {5,6}; lowest passes 100, 100, 90, 90."""
    img = np.array([[10, 100, 50, 200, 80, 90, 5]], dtype=np.uint8)
    L0, K = oracle.watershed(img, 4)
    assert L0.ravel().tolist() == [0, 0, 1, 1, 2, 3, 3]
    levels, counts = oracle.waterfall(L0, img, 4, 2)
    assert levels[0].ravel().tolist() == [0, 0, 0, 0, 1, 1, 1]


def test_kept_edges_are_lowest_passes():
    rng = np.random.default_rng(5)
    img = rng.integers(0, 8, size=(10, 10)).astype(np.uint8)
    L0, K = oracle.watershed(img, 4)
    levels, counts = oracle.waterfall(L0, img, 4, 2)
    L1 = levels[0]
    G = Grid(img.shape, 4)
    I = img.ravel().tolist()
    a0 = L0.ravel().tolist()
    a1 = L1.ravel().tolist()
    passes = {}
    for p in range(G.N):
        for q in G.nb(p):
            if a0[p] != a0[q]:
                key = (min(a0[p], a0[q]), max(a0[p], a0[q]))
                passes[key] = min(passes.get(key, 999), max(I[p], I[q]))
    newmin = {}
    for (a, b), h in passes.items():
        newmin[a] = min(newmin.get(a, 999), h)
        newmin[b] = min(newmin.get(b, 999), h)
    # every region of level 0 joins the region across its lowest pass
    first = {a0[p]: p for p in reversed(range(G.N))}
    for (a, b), h in passes.items():
        if h == newmin[a] or h == newmin[b]:
            assert a1[first[a]] == a1[first[b]]
