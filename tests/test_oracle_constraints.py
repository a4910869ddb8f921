"""Pins of the constraint oracle (oracle/constraints.py)."""
import numpy as np
import pytest

from oracle import constraints as K


def test_positivity_closed_forms():
    x = np.array([-2.0, -0.5, 0.0, 0.3, 1.5])
    np.testing.assert_array_equal(K.positivity(x, 1.0), [0.0, 0.0, 0.0, 0.3, 1.5])
    np.testing.assert_array_equal(K.positivity(x, 0.0), x)
    np.testing.assert_allclose(K.positivity(x, 0.25), [-1.5, -0.375, 0.0, 0.3, 1.5])


def test_rz_blur_closed_forms():
    rng = np.random.default_rng(0)
    const = np.full((7, 3, 4), 2.5)
    np.testing.assert_allclose(K.rz_blur(const, 1.3), const, rtol=1e-14)
    x = rng.standard_normal((6, 5, 4))
    np.testing.assert_allclose(K.rz_blur(x, 0.1), x, rtol=1e-12, atol=1e-14)  # taps at +-1 weigh e^-50
    np.testing.assert_array_equal(K.rz_blur(x, 1.0, 0.0), x)
    # reversing the slice order commutes with the blur
    np.testing.assert_allclose(K.rz_blur(x[::-1], 0.8)[::-1], K.rz_blur(x, 0.8), rtol=1e-13)
    # a delta in the middle of a deep volume spreads as the normalised Gaussian taps
    d = np.zeros((21, 1, 1))
    d[10] = 1.0
    y = K.rz_blur(d, 1.5)[:, 0, 0]
    t = np.exp(-0.5 * (np.arange(-10, 11) / 1.5) ** 2)
    t[np.abs(np.arange(-10, 11)) > 6] = 0.0
    # slices 6..14, whose 4-sigma window lies inside the volume: the plain normalised taps
    np.testing.assert_allclose(y[6:15], (t / t.sum())[6:15], rtol=1e-12, atol=1e-16)
    assert (y[:4] == 0).all() and (y[17:] == 0).all()


def test_rz_blur_matches_scipy_normalised_convolution():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(1)
    x = rng.standard_normal((9, 4, 5))
    for sigma in (0.7, 1.0, 2.2):
        num = ndimage.gaussian_filter1d(x, sigma, axis=0, mode="constant", cval=0.0, truncate=4.0)
        den = ndimage.gaussian_filter1d(np.ones_like(x), sigma, axis=0, mode="constant", cval=0.0, truncate=4.0)
        # scipy truncates at int(4 sigma + 0.5) taps; compare where that equals ceil(4 sigma)
        if int(4 * sigma + 0.5) == int(np.ceil(4 * sigma)):
            np.testing.assert_allclose(K.rz_blur(x, sigma), num / den, rtol=1e-10, atol=1e-12)


def test_constrain_order():
    rng = np.random.default_rng(2)
    phase = rng.standard_normal((5, 3, 3))
    amp = 1.0 + 0.1 * rng.standard_normal((5, 3, 3))
    a, p = K.constrain(amp, phase, positivity_relax=1.0, rz_sigma=1.0)
    assert (p >= 0).all()
    np.testing.assert_allclose(p, np.maximum(K.rz_blur(phase, 1.0), 0.0))
    np.testing.assert_allclose(a, K.rz_blur(amp, 1.0))
