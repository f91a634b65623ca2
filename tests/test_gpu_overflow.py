"""Fixed-point overflow on the GPU. Every image contribution is non-negative,
so a pixel whose sum passes 2^63 turns negative; the check after each run
finds it and flags MC_ERR_OVERFLOW. The photons here all land their camera
terms in a 1 x 1 image, and the fraction bits are chosen from a run at
F = 16 so that the same photons' sum at F lies in [2^63, 2^64); two fewer
bits keep it below 2^62 and must not be flagged."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LX, LY, LZ = 45.0, 10.0, 10.0
N_PHOTONS = 1_000_000


def _wrapping_bits(gpu, med, cam, geo):
    e = gpu.Engine(cam, geo)
    e.run(med, N_PHOTONS, seed=3, image_frac_bits=16)
    e.check()
    s16 = int(e.result()["raw_image"].sum())
    assert s16 > 0
    f = int(round(63.5 - math.log2(s16 * 2.0 ** -16)))
    assert 8 <= f <= 48, f
    assert 2.0 ** 63 <= s16 * 2.0 ** (f - 16) < 2.0 ** 64
    return f, s16


def test_a_pixel_sum_past_2_63_is_flagged(gpu):
    from paper_2507_23189_gb300 import _native as N
    med = gpu.Medium(5.0 / LX, 0.0, "hg", 0.0, None)
    cam, geo = gpu.Camera(1, 1, 16, 5 * 2 ** 0.5), gpu.Geometry(LX, LY, LZ)
    f, s16 = _wrapping_bits(gpu, med, cam, geo)
    e = gpu.Engine(cam, geo)
    e.run(med, N_PHOTONS, seed=3, image_frac_bits=f)
    with pytest.raises(N.McError) as err:
        e.check()
    assert err.value.status == -5
    assert int(e.image.cpu().numpy()[0, 0]) < 0        # the wrapped sum
    # the same photons with two fewer fraction bits: below 2^62, not flagged,
    # and the sum scales with 2^F up to the rounding of each contribution
    # (to 2^-16 weight units at F = 16, a few 1e-5 of the sum here)
    e.run(med, N_PHOTONS, seed=3, image_frac_bits=f - 2)
    e.check()
    s = int(e.result()["raw_image"].sum())
    assert 0 < s < 2 ** 62
    assert s == pytest.approx(s16 * 2.0 ** (f - 2 - 16), rel=1e-3)


def test_a_wrapped_medium_in_a_batch_is_flagged(gpu):
    from paper_2507_23189_gb300 import _native as N
    med = gpu.Medium(5.0 / LX, 0.0, "hg", 0.0, None)
    cam, geo = gpu.Camera(1, 1, 16, 5 * 2 ** 0.5), gpu.Geometry(LX, LY, LZ)
    f, _ = _wrapping_bits(gpu, med, cam, geo)
    b = gpu.Batch(2, cam, geo)
    b.run([med, med], [1000, N_PHOTONS], seeds=[1, 3], image_frac_bits=f)
    with pytest.raises(N.McError) as err:
        b.check()
    assert err.value.status == -5
    img = b.image.cpu().numpy()
    assert img[0, 0, 0] > 0 and img[1, 0, 0] < 0
    b.run([med, med], [1000, N_PHOTONS], seeds=[1, 3], image_frac_bits=f - 2)
    b.check()
    assert np.all(b.image.cpu().numpy() > 0)
