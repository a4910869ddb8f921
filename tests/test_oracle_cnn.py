"""Pins of the CNN oracle (oracle/cnn.py) against things other than itself: brute-force loops,
scipy's correlation, torch's bf16 conversion, closed forms, adjoint identities and finite
differences."""
import numpy as np
import pytest

from oracle import cnn as C


def _brute_conv(x, w, b, stride, up):
    """Direct six-fold loop over outputs, taps and channels on the upsampled, zero-padded grid."""
    B, H, W, IC = x.shape
    UH, UW = H * up, W * up
    OH, OW = (UH + stride - 1) // stride, (UW + stride - 1) // stride
    OC = w.shape[0]
    z = np.zeros((B, OH, OW, OC))
    for n in range(B):
        for oy in range(OH):
            for ox in range(OW):
                for o in range(OC):
                    acc = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            uy, ux = stride * oy + ky - 1, stride * ox + kx - 1
                            if 0 <= uy < UH and 0 <= ux < UW:
                                for c in range(IC):
                                    acc += w[o, ky, kx, c] * x[n, uy // up, ux // up, c]
                    z[n, oy, ox, o] = acc
    return z


@pytest.mark.parametrize("stride,up,H,W", [(1, 1, 5, 6), (2, 1, 5, 6), (2, 1, 6, 4), (1, 2, 3, 4), (1, 4, 2, 3)])
def test_conv_matches_brute_force(stride, up, H, W):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, H, W, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(C.conv_forward(x, w, b, stride, up), _brute_conv(x, w, b, stride, up),
                               rtol=1e-12, atol=1e-12)


def test_conv_matches_scipy_correlation():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 9, 7, 2))
    w = rng.standard_normal((3, 3, 3, 2))
    z = C.conv_forward(x, w, np.zeros(3), 1, 1)
    for o in range(3):
        ref = sum(signal.correlate2d(x[0, :, :, c], w[o, :, :, c], mode="same", boundary="fill") for c in range(2))
        np.testing.assert_allclose(z[0, :, :, o], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("stride,up", [(1, 1), (2, 1), (1, 2), (1, 4)])
def test_conv_backward_is_the_adjoint(stride, up):
    """<dz, conv(x, w)> is bilinear: its x, w, b gradients satisfy the dot-product identities."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 4, 6, 3))
    w = rng.standard_normal((5, 3, 3, 3))
    b = rng.standard_normal(5)
    z = C.conv_forward(x, w, b, stride, up)
    dz = rng.standard_normal(z.shape)
    dx, dw, db = C.conv_backward(x, w, stride, up, dz)
    lin_x = C.conv_forward(x, w, np.zeros(5), stride, up)
    assert np.isclose((dz * lin_x).sum(), (dx * x).sum(), rtol=1e-12)
    assert np.isclose((dz * lin_x).sum(), (dw * w).sum(), rtol=1e-12)
    assert np.isclose((dz * (z - lin_x)).sum(), (db * b).sum(), rtol=1e-12)


def test_upsample_block_sum_adjoint():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 3, 5, 2))
    y = rng.standard_normal((2, 12, 20, 2))
    assert np.isclose((C.upsample(x, 4) * y).sum(), (x * C.block_sum(y, 4)).sum(), rtol=1e-12)


def test_bf16_rounding():
    # ties to even at 1.0: spacing 2^-7
    assert C.bf16(1.0 + 2.0 ** -8) == 1.0
    assert C.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert C.bf16(-1.0 - 2.0 ** -8 - 2.0 ** -20) == -1.0 - 2.0 ** -7
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(5).standard_normal(10000) * 10.0 ** np.random.default_rng(6).uniform(-20, 20, 10000)
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(C.bf16(v), ref)


def test_param_count_and_shapes():
    assert C.param_count() == sum(9 * i * o + o for i, o, _, _, _ in C.LAYERS)
    assert 1.5e6 < C.param_count() < 2.5e6
    p = np.arange(C.param_count(), dtype=np.float64)
    np.testing.assert_array_equal(C.pack(C.unpack(p)), p)
    out, acts = C.forward(np.zeros(C.param_count()), np.zeros((1, 32, 32)), 0.2)
    assert out.shape == (1, 16, 16, 2) and len(acts) == 6


def test_mse_closed_form():
    """Zero weights and output bias beta: output = beta everywhere, loss = mean((beta - Y)^2),
    d loss / d beta_c = 2 mean over pixels (beta_c - Y_c) / 2."""
    p = np.zeros(C.param_count())
    p[-2:] = [0.5, -0.25]
    Y = np.zeros((2, 16, 16, 2))
    Y[..., 0] = 1.0
    loss, g = C.loss_and_grad(p, np.ones((2, 32, 32)), Y, 0.2, bf=False)
    assert np.isclose(loss, ((0.5 - 1.0) ** 2 + 0.25 ** 2) / 2)
    assert np.allclose(g[-2:], [2 * (0.5 - 1.0) / 2, 2 * (-0.25) / 2])


def _small_params(rng, scale=0.3):
    wb = []
    for ic, oc, _, _, _ in C.LAYERS:
        wb.append((rng.standard_normal((oc, 3, 3, ic)) * scale / np.sqrt(9 * ic), 0.05 * rng.standard_normal(oc)))
    return C.pack(wb)


def test_network_gradient_central_differences():
    rng = np.random.default_rng(7)
    p = _small_params(rng, scale=1.5)
    I = rng.gamma(2.0, 30.0, (2, 32, 32))
    Y = 0.1 * rng.standard_normal((2, 16, 16, 2))
    loss, g = C.loss_and_grad(p, I, Y, 0.2, bf=False)
    # entries from every layer's weights and biases
    offs, o = [], 0
    for ic, oc, _, _, _ in C.LAYERS:
        offs += [o + int(rng.integers(9 * ic * oc)), o + 9 * ic * oc + int(rng.integers(oc))]
        o += 9 * ic * oc + oc
    for k in offs:
        h = 1e-5
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (C.loss_and_grad(pp, I, Y, 0.2, bf=False)[0] - C.loss_and_grad(pm, I, Y, 0.2, bf=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3 * np.abs(g).max()), (k, fd, g[k])


def test_bf16_emulation_is_close_to_exact():
    rng = np.random.default_rng(8)
    p = _small_params(rng, scale=1.5)
    I = rng.gamma(2.0, 30.0, (2, 32, 32))
    Y = 0.1 * rng.standard_normal((2, 16, 16, 2))
    l0, g0 = C.loss_and_grad(p, I, Y, 0.2, bf=False)
    l1, g1 = C.loss_and_grad(p, I, Y, 0.2, bf=True)
    assert abs(l1 - l0) <= 2e-2 * l0
    assert np.linalg.norm(g1 - g0) <= 5e-2 * np.linalg.norm(g0)


def test_targets_stitch_and_nmse():
    rng = np.random.default_rng(9)
    Nz, H, W, N = 3, 40, 44, 16
    phase = rng.uniform(0, 0.3, (Nz, H, W))
    amp = np.exp(-rng.uniform(0, 0.1, (Nz, H, W)))
    corners = [(0, 0), (4, 8), (20, 24), (24, 28)]
    Y = C.targets(amp, phase, corners, N)
    assert Y.shape == (4, 8, 8, 2)
    assert np.allclose(Y[1, 0, 0, 0], phase[:, 4 + 4, 8 + 4].sum())
    assert np.allclose(Y[2, 7, 7, 1], np.log(amp[:, 20 + 4 + 7, 24 + 4 + 7]).sum())
    # stitching the exact targets reproduces the depth sums where covered (any positive weight)
    wgt = rng.uniform(0.5, 1.0, (8, 8))
    a0, p0 = C.stitch(Y, corners, wgt, H, W, N, Nz)
    phi = phase.sum(0)
    assert np.allclose(p0.sum(0)[8:12, 12:16], phi[8:12, 12:16])
    assert np.allclose(np.log(a0).sum(0)[8:12, 12:16], np.log(amp).sum(0)[8:12, 12:16])
    assert np.all(p0[:, 0:4, :] == 0) and np.all(a0[:, 0:4, :] == 1)
    roi = (4, 36, 4, 40)
    assert C.nmse(phi, phi, roi) == 0.0
    assert np.isclose(C.nmse(np.zeros_like(phi), phi, roi), 1.0)
    assert np.isclose(C.nmse(phi + 3.0, phi, roi), 0.0, atol=1e-20)
