"""Pins of the oracle (and of the literal simulators) to the worked examples
the paper prints: Sec. 3.3 (synchronous step II on 75, 89 x 2n, 81), Sec. 3.4
(Alg. 3 on the 14 x 1 image, blocks of 3), Fig. 4 (path reduction rounds) and
the 1D property of Sec. 3.1."""
import math

import numpy as np
import pytest

import oracle
from brute import literal_alg1, literal_bal_1d, step3_rounds, canonical
from conftest import read_golden


def test_sec33_step1_states():
    g = read_golden("sec33_plateau_2n.txt")
    img = np.array([g["values"]], dtype=np.uint8)
    S, L = oracle.step1(img, 4)
    assert S.ravel().tolist() == g["states_step1"]


@pytest.mark.parametrize("n", [2, 3, 5, 8, 13])
def test_sec33_general_n(n):
    vals = [75] + [89] * (2 * n) + [81]
    img = np.array([vals], dtype=np.uint8)
    S, _ = oracle.step1(img, 4)
    assert S.ravel().tolist() == [1, 0] + [2] * (2 * n - 2) + [0, 1]
    dist = oracle.plateau_distance(img, 4).ravel().tolist()
    # distance from the nearer end of the plateau
    assert dist[1:-1] == [min(i, 2 * n - 1 - i) for i in range(2 * n)]
    labels, K = oracle.watershed(img, 4)
    assert K == 2
    assert labels.ravel().tolist() == [0] * (n + 1) + [1] * (n + 1)
    # literal synchronous simulation: n iterations of step II
    _, tr = literal_alg1(img, 4, return_trace=True)
    assert tr["it2"] == n


def test_sec33_arrows_and_split():
    g = read_golden("sec33_plateau_2n.txt")
    img = np.array([g["values"]], dtype=np.uint8)
    labels, K, S1, dist, ptr = oracle.watershed(img, 4, debug=True)
    assert ptr.ravel().tolist() == g["arrows_step2"]
    assert labels.ravel().tolist() == g["basins"]
    _, tr = literal_alg1(img, 4, return_trace=True)
    assert tr["it2"] == g["step2_iterations"]
    assert tr["L2"] == g["arrows_step2"]


def test_sec33_states_after_n_minus_2_iterations():
    """Replays the synchronous rounds and checks the printed intermediate state."""
    g = read_golden("sec33_plateau_2n.txt")
    n = g["n"]
    vals = g["values"]
    S = list(g["states_step1"])
    for _ in range(n - 2):
        Sn = list(S)
        for p in range(len(vals)):
            if S[p] >= 2 and any(0 <= q < len(vals) and S[q] == 0 and vals[q] == vals[p]
                                 for q in (p - 1, p + 1)):
                Sn[p] = 0
        S = Sn
    assert S == g["states_after_n_minus_2"]
    # the oracle's distances say the same thing: distance <= n-2 <=> state 0
    dist = oracle.plateau_distance(np.array([vals], dtype=np.uint8), 4).ravel().tolist()
    assert [0 if (d >= 0 and d <= n - 2) else s for d, s in zip(dist, g["states_step1"])] == S


def test_sec34_balanced_example():
    g = read_golden("sec34_balanced_14.txt")
    hist = literal_bal_1d(g["values"], g["block"])
    assert len(hist) == 3
    assert hist[0] == g["global_iteration_1"]
    assert hist[1] == g["global_iteration_2"]
    assert hist[2] == g["global_iteration_3"]
    img = np.array([g["values"]], dtype=np.uint8)
    dist = oracle.plateau_distance(img, 4).ravel().tolist()
    assert dist[1:13] == g["distances"]
    # fixpoint of Alg. 3 = -distance on the plateau
    assert [-s for s in hist[-1][1:13]] == g["distances"]
    labels, K = oracle.watershed(img, 4)
    assert labels.ravel().tolist() == [0] * 7 + [1] * 7


def test_fig4_path_reduction_rounds():
    g = read_golden("fig4_path_reduction.txt")
    n = g["path_length"]
    L = [min(i + 1, n) for i in range(n + 1)]   # 0 -> 1 -> ... -> n (self loop)
    rounds, final = step3_rounds(L, g["RR"])
    assert rounds - 1 == g["iterations"] == math.ceil(math.log(n, g["RR"] + 1))
    assert final == [n] * (n + 1)
    # the oracle's root chase gives the same roots on a 1D descending ramp
    img = np.array([list(range(n, -1, -1))], dtype=np.uint8)
    roots = oracle.roots_without_merge(img, 4).ravel().tolist()
    assert roots == [n] * (n + 1)


@pytest.mark.parametrize("seed", range(40))
def test_1d_property(seed):
    """Sec. 3.1: in 1D, steps I-III already give the watershed, and the only
    state-3 pixel of a minimal plateau is its rightmost pixel."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    img = rng.integers(0, 4, size=(1, n)).astype(np.uint8)
    S, _ = oracle.step1(img, 4)
    roots = oracle.roots_without_merge(img, 4)
    labels, K = oracle.watershed(img, 4)
    assert np.array_equal(canonical(roots), labels)
    v = img.ravel().tolist()
    s = S.ravel().tolist()
    for p in range(n):
        if s[p] == 3:
            # rightmost pixel of an equal run, with nothing lower adjacent to the run
            assert p == n - 1 or v[p + 1] != v[p]
            assert p > 0 and v[p - 1] == v[p]
