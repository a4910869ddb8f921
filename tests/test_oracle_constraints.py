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


# --- k_z filter (Eq. 10-12) -------------------------------------------------------------------

SHAPE, DX, DZ = (8, 12, 16), 0.5, 2.0


def _wave(a, b, c):
    """cos(2 pi (c z / Nz + b y / H + a x / W)): a real eigenfunction of every even 3D filter."""
    Nz, H, W = SHAPE
    z, y, x = np.meshgrid(np.arange(Nz), np.arange(H), np.arange(W), indexing="ij")
    return np.cos(2 * np.pi * (c * z / Nz + b * y / H + a * x / W))


def test_kz_filter_identity_and_constants():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(SHAPE)
    np.testing.assert_allclose(K.kz_filter(x, DX, DZ, 0.0, 0.0), x, atol=1e-13)  # W = 1
    const = np.full(SHAPE, 1.7)
    np.testing.assert_allclose(K.kz_filter(const, DX, DZ, 1.0, 3.0), const, rtol=1e-13)  # W(0) = 1
    np.testing.assert_array_equal(K.kz_filter(x, DX, DZ, 1.0, 0.5, r=0.0), x)
    full = K.kz_filter(x, DX, DZ, 1.0, 0.5)
    np.testing.assert_allclose(K.kz_filter(x, DX, DZ, 1.0, 0.5, r=0.5), 0.5 * (x + full), rtol=1e-13, atol=1e-15)


def test_kz_filter_closed_values_on_plane_waves():
    Nz, H, W = SHAPE
    # lateral wave (k_z = 0): the arctan term vanishes whatever beta; alpha chosen so that
    # exp(-alpha k_y^2) = 1/2
    ky = 2 / (H * DX)
    x = _wave(0, 2, 0)
    np.testing.assert_allclose(K.kz_filter(x, DX, DZ, 5.0, np.log(2) / ky ** 2), 0.5 * x, atol=1e-13)
    # beta^2 k_z^2 = k_x^2 + eps: arctan(1) = pi / 4, W = 1/2
    kx, kz = 3 / (W * DX), 1 / (Nz * DZ)
    beta = np.sqrt((kx ** 2 + K.KZ_EPS) / kz ** 2)
    x = _wave(3, 0, 1)
    np.testing.assert_allclose(K.kz_filter(x, DX, DZ, beta, 0.0), 0.5 * x, atol=1e-13)
    # axial wave (k_r = 0), beta^2 k_z^2 = sqrt(3) eps: arctan(sqrt 3) = pi / 3, W = 1/3
    kz = 2 / (Nz * DZ)
    beta = np.sqrt(np.sqrt(3) * K.KZ_EPS) / kz
    x = _wave(0, 0, 2)
    np.testing.assert_allclose(K.kz_filter(x, DX, DZ, beta, 0.0), x / 3, atol=1e-13)


def test_kz_filter_is_periodic_in_depth():
    """Circular shifts commute with the filter (the wrap-around of a periodic 3D DFT)."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal(SHAPE)
    y = K.kz_filter(x, DX, DZ, 1.0, 0.2)
    np.testing.assert_allclose(K.kz_filter(np.roll(x, 3, axis=0), DX, DZ, 1.0, 0.2), np.roll(y, 3, axis=0),
                               atol=1e-13)
    np.testing.assert_allclose(K.kz_filter(np.roll(x, -5, axis=2), DX, DZ, 1.0, 0.2), np.roll(y, -5, axis=2),
                               atol=1e-13)


def test_constrain_order_with_kz_filter():
    rng = np.random.default_rng(5)
    amp = 1.0 + 0.1 * rng.standard_normal(SHAPE)
    phase = rng.standard_normal(SHAPE)
    a, p = K.constrain(amp, phase, positivity_relax=1.0, rz_sigma=1.0, kz_beta=1.0, kz_alpha=0.1, kz_relax=0.7,
                       dx=DX, dz=DZ)
    np.testing.assert_allclose(a, K.rz_blur(K.kz_filter(amp, DX, DZ, 1.0, 0.1, 0.7), 1.0))
    np.testing.assert_allclose(p, np.maximum(K.rz_blur(K.kz_filter(phase, DX, DZ, 1.0, 0.1, 0.7), 1.0), 0.0))


# --- probe-mode orthogonalisation --------------------------------------------------------------

def _modes(M, N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((M, N, N)) + 1j * rng.standard_normal((M, N, N))


def test_orthogonalize_matches_svd():
    P = _modes(5, 6, 6)
    Q, lam = K.orthogonalize_probe(P)
    A = P.reshape(5, -1)
    _, sv, Vh = np.linalg.svd(A, full_matrices=False)
    np.testing.assert_allclose(lam, sv ** 2, rtol=1e-12)
    S = sv[:, None] * Vh  # the SVD's modes, each up to a phase
    Qf = Q.reshape(5, -1)
    for k in range(5):
        ph = np.vdot(S[k], Qf[k])
        assert np.isclose(abs(ph), sv[k] ** 2, rtol=1e-12)
        np.testing.assert_allclose(Qf[k], S[k] * ph / abs(ph), atol=1e-11)


def test_orthogonalize_invariants():
    P = _modes(4, 5, 7)
    Q, lam = K.orthogonalize_probe(P)
    A, B = P.reshape(4, -1), Q.reshape(4, -1)
    np.testing.assert_allclose(B.conj().T @ B, A.conj().T @ A, atol=1e-11)  # the density matrix
    np.testing.assert_allclose(B @ B.conj().T, np.diag(lam), atol=1e-11)  # orthogonal, powers lam
    assert (np.diff(lam) <= 0).all()


def test_orthogonalize_fixed_points():
    # orthogonal modes come back sorted by power and unchanged (U is a permutation)
    N = 4
    P = np.zeros((3, N, N), dtype=complex)
    P[0, 0, 0], P[1, 1, 2], P[2, 3, 3] = 0.5j, 2.0, -1.0 + 1.0j
    Q, lam = K.orthogonalize_probe(P)
    np.testing.assert_array_equal(Q, P[[1, 2, 0]])
    np.testing.assert_allclose(lam, [4.0, 2.0, 0.25])
    one = _modes(1, 5, 8)
    np.testing.assert_allclose(K.orthogonalize_probe(one)[0], one, rtol=1e-15)


def test_orthogonalize_phase_convention():
    """Each new mode is sum_m c_km P_m with the largest |c_km| real and positive (reading C5)."""
    P = _modes(4, 6, 9)
    Q, _ = K.orthogonalize_probe(P)
    A, B = P.reshape(4, -1), Q.reshape(4, -1)
    C = B @ np.linalg.pinv(A)  # B = C A, C = U^H
    for k in range(4):
        m = int(np.argmax(np.abs(C[k])))
        assert abs(C[k, m].imag) <= 1e-12 * abs(C[k, m]) and C[k, m].real > 0
