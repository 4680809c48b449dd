"""The CPU oracle over many inputs at once, in worker processes.

Full-size parity cases (hundreds of images) would take minutes on one core.
The workers are started with the "spawn" method, so they inherit no CUDA
state of the test process, and import only numpy and the oracle.  Each worker
returns, per input, the oracle's region counts and the SHA-256 digest of its
label planes; the test compares those with the digest of the GPU's planes,
and recomputes the oracle in-process for any input whose digests differ, to
report the first differing element.
"""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os

import numpy as np


def digest(levels) -> str:
    """SHA-256 of int32 label planes (numpy array or CPU torch tensor)."""
    a = np.ascontiguousarray(np.asarray(levels), dtype=np.int32)
    return hashlib.sha256(a.tobytes()).hexdigest()


def _segment_digest(args):
    import oracle
    arr, conn, NL = args
    levels, counts = oracle.segment(arr, conn, NL)
    return [int(c) for c in counts], digest(levels)


def first_difference(got: np.ndarray, want: np.ndarray) -> str:
    """Where two label arrays of one shape first differ, as text."""
    bad = np.argwhere(got != want)
    if bad.size == 0:
        return "no element differs"
    idx = tuple(int(v) for v in bad[0])
    return f"{len(bad)} elements differ, first at {idx}: got {int(got[idx])}, oracle {int(want[idx])}"


class OraclePool:
    """A spawned pool that runs oracle.segment over (array, conn, NL) items."""

    def __init__(self, workers: int | None = None):
        n = workers or min(16, os.cpu_count() or 1)
        self.pool = mp.get_context("spawn").Pool(n)

    def segment_digests(self, items):
        """[(counts, digest)] in the order of items."""
        return self.pool.map(_segment_digest, items, chunksize=1)

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.pool.terminate()
        self.pool.join()
