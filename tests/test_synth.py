"""The seeded input generators (not the method): SplitMix64 against its
published first outputs, the C squared-EDT against brute force."""
import numpy as np
import pytest

from paper_2410_08946_gb300 import synth


def test_splitmix64_published_outputs():
    # first two outputs of SplitMix64 started from state 0
    out = synth.splitmix64(np.array([0, 0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_uniform_ranges_and_determinism():
    a = synth.uniform(1, 2, 1000, 4.0, 20.0)
    b = synth.uniform(1, 2, 1000, 4.0, 20.0)
    assert np.array_equal(a, b) and a.min() >= 4.0 and a.max() < 20.0
    k = synth.integers(5, 6, 5000, 0, 16)
    assert k.min() == 0 and k.max() == 16


@pytest.mark.parametrize("shape,n", [((5, 7, 9), 3), ((11, 6, 8), 9), ((1, 13, 17), 4), ((16, 16, 16), 1)])
def test_distance_volume_matches_bruteforce(shape, n):
    D, H, W = shape
    got = synth.distance_volume(D, H, W, n, seed=99)
    ref = synth.distance_volume_reference(D, H, W, n, seed=99)
    assert np.array_equal(got, ref)


def test_blob_image_shape_and_range():
    img = synth.blob_image(64, 80, 12, seed=7)
    assert img.shape == (64, 80) and img.dtype == np.uint8
    assert img.max() > 40
    assert np.array_equal(img, synth.blob_image(64, 80, 12, seed=7))


def test_batch_shapes_range():
    shp = synth.batch_shapes(512, 64, 2048, seed=3)
    sides = np.array(shp).ravel()
    assert sides.min() >= 64 and sides.max() <= 2048


def test_request_stream_rate():
    reqs = synth.request_stream(200.0, 10.0, seed=4)
    assert 1700 < len(reqs) < 2300
    frac3 = np.mean([r["kind"] == "3d" for r in reqs])
    assert 0.15 < frac3 < 0.25
