"""Pins of the oracle's 3D gradient (the 2D pipeline steps of Sec. 1, smooth
then gradient magnitude, on a volume: 5x5x5 binomial blur, 3x3x3 Sobel, exact
floor square root, >> shift, clip to 65535; replicated borders).

Closed forms: a constant volume has gradient 0; on a linear ramp
a x + b y + c z the blur is the identity away from the border and the Sobel
sums are 32 a, 32 b, 32 c, so the magnitude is floor(32 sqrt(a^2+b^2+c^2)).
Consistency with the pinned 2D operator: on a volume constant along z the 3D
blur equals the 2D blur and (gx, gy, gz) = (4 gx2, 4 gy2, 0), so
floor(sqrt(16 s)) >> 2 = floor(sqrt(s)), the 2D magnitude before its clip.
Symmetries: permuting the axes or mirroring the volume permutes / mirrors the
result (an axis or sign mix-up breaks one of them)."""
import numpy as np
import pytest

import oracle


def test_constant_is_zero():
    for dt in (np.uint8, np.uint16):
        assert not oracle.gradient3d(np.full((5, 6, 7), 200, dtype=dt)).any()


@pytest.mark.parametrize("a,b,c", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (3, 2, 1), (5, 7, 11), (40, 0, 30)])
def test_linear_ramp_interior(a, b, c):
    D, H, W = 11, 12, 13
    z, y, x = np.indices((D, H, W))
    v = (a * x + b * y + c * z + 100).astype(np.uint16)
    g = oracle.gradient3d(v)
    want = int(np.floor(32 * np.sqrt(a * a + b * b + c * c)))
    assert np.all(g[3:-3, 3:-3, 3:-3] == want)
    assert np.all(oracle.gradient3d(v, shift=2)[3:-3, 3:-3, 3:-3] == want >> 2)


def test_matches_2d_operator_on_z_constant_volumes():
    rng = np.random.default_rng(0)
    for trial in range(4):
        H, W = rng.integers(5, 40, size=2)
        u = (rng.integers(0, 60, size=(H, W))).astype(np.uint8)   # small values: no 2D clip at 255
        v = np.repeat(u[None], 6, axis=0)
        g3 = oracle.gradient3d(v)
        g2 = oracle.gradient2d(u)
        assert np.all(g2 < 255)
        for zz in range(6):
            assert np.array_equal(g3[zz] >> 2, g2.astype(np.uint16))


def test_axis_permutations_and_mirrors():
    rng = np.random.default_rng(1)
    v = rng.integers(0, 65535, size=(9, 9, 9)).astype(np.uint16)
    g = oracle.gradient3d(v)
    for perm in [(0, 2, 1), (1, 0, 2), (2, 1, 0), (1, 2, 0)]:
        assert np.array_equal(oracle.gradient3d(np.ascontiguousarray(v.transpose(perm))), g.transpose(perm))
    for ax in range(3):
        assert np.array_equal(oracle.gradient3d(np.ascontiguousarray(np.flip(v, ax))), np.flip(g, ax))
    # non-cubic shapes too
    w = rng.integers(0, 255, size=(4, 7, 10)).astype(np.uint8)
    assert np.array_equal(oracle.gradient3d(np.ascontiguousarray(w.transpose(2, 1, 0))),
                          oracle.gradient3d(w).transpose(2, 1, 0))


def test_clip_and_shift():
    v = np.zeros((7, 7, 7), dtype=np.uint16)
    v[:, :, 4:] = 65535   # a step: huge gradient at the interface
    g = oracle.gradient3d(v)
    assert g.max() == 65535
    assert oracle.gradient3d(v, shift=8).max() < 65535


def test_tiny_volumes():
    assert oracle.gradient3d(np.array([[[7]]], dtype=np.uint8)).tolist() == [[[0]]]
    v = np.arange(8, dtype=np.uint16).reshape(2, 2, 2) * 1000
    g = oracle.gradient3d(v)
    assert g.shape == (2, 2, 2) and np.array_equal(g, g[::-1, ::-1, ::-1])   # point symmetry of a ramp
