"""Pins of the oracle's gradient stage (a0) by closed forms.  The paper only
says "Gaussian blur, then gradient magnitude" (Sec. 1, Fig. 1, Fig. 2), so the
operator is this build's reading: 5x5 binomial blur with round-half-up, 3x3
integer Sobel, exact floor square root, clip to 255, optional >> shift.
Parity pinned by definition only (no paper values exist)."""
import math

import numpy as np
import pytest

import oracle

W5 = [1, 4, 6, 4, 1]


def test_isqrt_against_math_isqrt():
    rng = np.random.default_rng(0)
    vals = list(range(0, 5000)) + [int(v) for v in rng.integers(0, 2 * 1020 * 1020 + 1, 20000)]
    for r in range(0, 1443):
        vals += [r * r - 1, r * r, r * r + 1]
    vals += [2**32 - 1, 2**40 + 12345, 2**62 - 1]
    for v in vals:
        if v >= 0:
            assert oracle.isqrt(v) == math.isqrt(v), v


def test_constant_image_zero_gradient():
    for v in (0, 77, 255):
        g = oracle.gradient2d(np.full((9, 13), v, dtype=np.uint8))
        assert not g.any()


@pytest.mark.parametrize("a,b", [(1, 0), (3, 0), (0, 5), (3, 4), (5, 12), (7, 7), (31, 0)])
def test_linear_ramp_closed_form(a, b):
    """On a linear ramp a*x + b*y the binomial blur is exact in the interior
    and Sobel gives gx = 8a, gy = 8b, so mag = floor(8 * sqrt(a^2 + b^2))."""
    H = W = 8 if a + b > 20 else 14
    y, x = np.mgrid[0:H, 0:W]
    img = a * x + b * y
    img = img - img.min()
    assert img.max() <= 255
    g = oracle.gradient2d(img.astype(np.uint8))
    want = min(255, math.isqrt(64 * (a * a + b * b)))
    assert (g[3:-3, 3:-3] == want).all()


def test_impulse_blur_then_sobel():
    """A single bright pixel: the blurred image is the binomial kernel scaled
    by v/256 (round half up); Sobel of that at the centre is 0 by symmetry and
    at (0, +1) is the horizontal difference of the kernel columns."""
    H = W = 15
    img = np.zeros((H, W), dtype=np.uint8)
    img[7, 7] = 200
    g = oracle.gradient2d(img)
    blur = np.zeros((H + 4, W + 4), dtype=np.int64)
    for i in range(5):
        for j in range(5):
            blur[7 + i, 7 + j] = (W5[i] * W5[j] * 200 + 128) >> 8
    b = blur[2:-2, 2:-2]          # blurred image on the H x W grid
    assert g[7, 7] == 0
    for (yy, xx) in [(7, 8), (6, 7), (5, 9), (9, 4)]:
        gx = (b[yy - 1, xx + 1] + 2 * b[yy, xx + 1] + b[yy + 1, xx + 1]) - \
             (b[yy - 1, xx - 1] + 2 * b[yy, xx - 1] + b[yy + 1, xx - 1])
        gy = (b[yy + 1, xx - 1] + 2 * b[yy + 1, xx] + b[yy + 1, xx + 1]) - \
             (b[yy - 1, xx - 1] + 2 * b[yy - 1, xx] + b[yy - 1, xx + 1])
        assert g[yy, xx] == min(255, math.isqrt(int(gx * gx + gy * gy)))


def test_symmetries():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, size=(17, 23)).astype(np.uint8)
    g = oracle.gradient2d(img)
    assert np.array_equal(oracle.gradient2d(np.ascontiguousarray(img.T)), g.T)
    assert np.array_equal(oracle.gradient2d(np.ascontiguousarray(img[::-1, ::-1])), g[::-1, ::-1])
    assert np.array_equal(oracle.gradient2d(np.ascontiguousarray(img[:, ::-1])), g[:, ::-1])


def test_quantisation_is_shift():
    rng = np.random.default_rng(4)
    img = rng.integers(0, 256, size=(31, 29)).astype(np.uint8)
    g0 = oracle.gradient2d(img, 0)
    for s in range(1, 8):
        assert np.array_equal(oracle.gradient2d(img, s), g0 >> s)


def test_saturates_at_255():
    img = np.zeros((12, 12), dtype=np.uint8)
    img[:, 6:] = 255
    g = oracle.gradient2d(img)
    assert g.max() == 255


def test_tiny_images_replicate_border():
    """A 1 x n image: the replicated rows give the blur a vertical weight of
    16 and make gy = 0, so mag(x) = 4 |b(x+1) - b(x-1)| with clamped x."""
    v = [0, 0, 0, 100, 100, 100, 30]
    n = len(v)
    cl = lambda i: min(max(i, 0), n - 1)
    b = [(16 * sum(W5[j + 2] * v[cl(x + j)] for j in range(-2, 3)) + 128) >> 8 for x in range(n)]
    want = [min(255, 4 * abs(b[cl(x + 1)] - b[cl(x - 1)])) for x in range(n)]
    g = oracle.gradient2d(np.array([v], dtype=np.uint8))
    assert g.ravel().tolist() == want
    assert oracle.gradient2d(np.array([[9]], dtype=np.uint8))[0, 0] == 0
