"""Pins for the oracle's image comparison metrics (Sec. 3.1.4 normalisation,
Table 3 RMSE and r, Table 4 radial zones): hand-worked small images, numpy's
corrcoef, invariances, and ring geometry counted by hand."""
import math

import numpy as np
import pytest

from oracle import metrics as M


def test_normalise_range_and_affine_invariance():
    rng = np.random.default_rng(1)
    a = rng.integers(-1000, 10**9, size=(17, 23))
    n = M.normalise(a)
    assert n.min() == 0.0 and n.max() == 1.0
    np.testing.assert_allclose(M.normalise(7 * a + 12345), n, rtol=0, atol=1e-15)
    assert np.all(M.normalise(np.full((3, 4), 9)) == 0.0)


def test_rmse_and_r_hand_example():
    ref = np.array([[0, 1], [2, 3]])
    a = np.array([[3, 2], [1, 0]])
    na, nr = M.normalise(a), M.normalise(ref)
    # normalised: ref (0, 1/3, 2/3, 1), a (1, 2/3, 1/3, 0): squared errors
    # (1, 1/9, 1/9, 1), mean 5/9
    assert M.rmse(na, nr) == pytest.approx(math.sqrt(5 / 9), rel=1e-15)
    assert M.pearson(na, nr) == pytest.approx(-1.0, rel=1e-15)


def test_pearson_is_numpy_corrcoef():
    rng = np.random.default_rng(2)
    a, b = rng.normal(size=500), rng.normal(size=500) + 0.3 * np.arange(500) / 500
    assert M.pearson(a, b) == pytest.approx(np.corrcoef(a, b)[0, 1], rel=1e-12)
    assert M.pearson(a, 2 * a + 3) == pytest.approx(1.0, rel=1e-14)
    assert M.pearson(a, np.ones_like(a)) == 0.0


def test_rings_of_a_4x4_image():
    # pixel centres at +-0.5, +-1.5: radii sqrt(0.5) (4 pixels), sqrt(2.5)
    # (8), sqrt(4.5) (4); rho_max = sqrt(8); three rings of width sqrt(8)/3
    ring = M.ring_index(4, 4, 3)
    want = np.array([[2, 1, 1, 2], [1, 0, 0, 1], [1, 0, 0, 1], [2, 1, 1, 2]])
    np.testing.assert_array_equal(ring, want)
    # f = rho^2 normalised: (rho^2 - 0.5) / 4 -> ring means 0, 0.5, 1
    f = np.array([[4.5, 2.5, 2.5, 4.5], [2.5, 0.5, 0.5, 2.5], [2.5, 0.5, 0.5, 2.5], [4.5, 2.5, 2.5, 4.5]])
    prof, cnt = M.radial_profile(M.normalise(f), 3)
    np.testing.assert_array_equal(cnt, [4, 8, 4])
    np.testing.assert_allclose(prof, [0.0, 0.5, 1.0], rtol=0, atol=1e-15)


def test_rectangular_image_rings_cover_every_pixel():
    ring = M.ring_index(10, 30, 8)
    assert ring.min() == 0 and ring.max() == 7
    # corners sit at the largest radius, the centre at the smallest
    assert ring[0, 0] == ring[-1, -1] == 7
    assert ring[4:6, 14:16].max() == 0


def test_zones():
    np.testing.assert_array_equal(M.zone_of_ring(6), [0, 1, 1, 1, 2, 2])
    np.testing.assert_array_equal(M.zone_of_ring(12), [0, 0] + [1] * 6 + [2] * 4)


def test_compare_identical_and_better_share():
    rng = np.random.default_rng(3)
    ref = rng.integers(0, 10**6, size=(40, 60))
    out = M.compare(ref, ref.copy(), 10**6 - ref, n_r=8)
    assert out[0] == 0.0 and out[1] == pytest.approx(1.0, rel=1e-14)
    assert np.all(out[2:5] == 0.0) and out[5] == pytest.approx(1.0, rel=1e-14)
    assert out[7] == pytest.approx(-1.0, rel=1e-14)
    assert out[12] == 1.0            # a equals ref on every ring, b does not
    assert out.size == M.N_OUT_FIXED + 3 * 8
    np.testing.assert_array_equal(out[13:21], out[21:29])
    single = M.compare(ref, ref, None, n_r=8)
    assert np.all(single[6:13] == 0.0) and np.all(single[29:] == 0.0)


def test_better_share_counts_only_rings_with_pixels():
    """Hand-worked 2 x 2 case: every pixel centre lies at half the
    half-diagonal, so with 4 rings only ring 2 holds pixels. Normalised, ref
    and a average 1/2 there and b averages 3/4: a is closer on the one ring
    that has pixels, a share of 1 (not 1/4), and the empty rings stay 0."""
    ref = np.array([[0, 1], [1, 0]])
    b = np.array([[0, 1], [1, 1]])
    out = M.compare(ref, ref.copy(), b, n_r=4)
    assert out[12] == 1.0
    np.testing.assert_array_equal(out[13:17], [0.0, 0.0, 0.5, 0.0])       # profile of ref
    np.testing.assert_array_equal(out[21:25], [0.0, 0.0, 0.75, 0.0])      # profile of b
