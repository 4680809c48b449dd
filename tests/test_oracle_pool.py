"""The spawned oracle pool used by the many-image full-size parity tests
returns the same counts and label digests as in-process oracle calls, in
input order, and the digest tells label planes apart."""
import numpy as np

import oracle
from oracle_pool import OraclePool, digest, first_difference
from paper_2410_08946_gb300 import synth


def test_pool_matches_in_process():
    items = [(oracle.gradient2d(synth.blob_image(40 + 7 * i, 33 + 5 * i, 6, seed=900 + i)), 4 if i % 2 else 8, 3)
             for i in range(5)]
    items.append((synth.distance_volume(9, 11, 13, 5, seed=901), 6, 4))
    with OraclePool(workers=2) as pool:
        got = pool.segment_digests(items)
    for (arr, conn, NL), (counts, dg) in zip(items, got):
        levels, want = oracle.segment(arr, conn, NL)
        assert counts == want.tolist()
        assert dg == digest(levels)


def test_digest_and_difference():
    a = np.arange(24, dtype=np.int32).reshape(2, 3, 4)
    b = a.copy()
    assert digest(a) == digest(b)
    b[1, 2, 3] = -1
    assert digest(a) != digest(b)
    assert "first at (1, 2, 3)" in first_difference(b, a)
