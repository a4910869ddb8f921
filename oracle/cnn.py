"""FP64 CPU oracle of the learned initialiser: a small convolutional encoder-decoder that maps a
log-scaled diffraction pattern to the object patch under the probe, its training gradient, and
the stitching of predicted patches into an initial object.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the CPU-baseline leg of the
benchmark; the product path never calls it.

The paper starts every reconstruction from a flat object (amplitude 1, phase U[0, 1e-8]; Sec.
"Preprocessing and initialization") and mentions learned direct solvers only as related work
(Sec. "Introduction").  The network here is this project's own initialiser; nothing in the paper
fixes its architecture, so the oracle is its definition written out:

  input   x0 = bf16(s_in * log(1 + I))                      I: [B, N, N] DC-centred pattern
  layer l z_l = conv3x3(up_l(a_{l-1}); stride_l) + b_l       zero padding 1 on the upsampled grid
          a_l = bf16(relu(z_l)) for l < 6;  output = z_6     (FP32 on the GPU, not rounded)
  loss    L = mean((output - Y)^2)                           Y: [B, N/2, N/2, 2] targets

  layer      in -> out channels   stride   nearest upsampling before the conv
  1          1 -> 48              2        1
  2          48 -> 96             2        1
  3          96 -> 192            2        1
  4          192 -> 384           2        1
  5          384 -> 256           1        2
  6          256 -> 2             1        4

Activations are [B, H, W, C] (channels last).  Weights are stored [OC, 3, 3, IC] followed by the
bias [OC], layer after layer, in one flat FP32 parameter vector.

bf16 storage (the kernels' operand precision) is emulated at the same points when `bf16=True`:
the input, every weight, every stored activation, and every activation gradient that feeds a
GEMM (dL/dz_l after its ReLU mask; dL/dz_6 from the loss).  Sums are exact in FP64 here and FP32
on the GPU, so the two agree to FP32 rounding except where that rounding moves a value across a
bf16 rounding boundary.

Pins (tests/test_oracle_cnn.py): brute-force loops on tiny convolutions (stride 1 and 2,
upsampling), scipy's 2D correlation as a library special case, torch's bf16 conversion, closed
forms (bf16 ties, MSE on constants, NMSE of the exact and of the zero estimate), adjoint
(dot-product) identities, and central finite differences of the full network gradient.
"""
from __future__ import annotations

import numpy as np

# (in_channels, out_channels, stride, upsample, relu)
LAYERS = (
    (1, 48, 2, 1, True),
    (48, 96, 2, 1, True),
    (96, 192, 2, 1, True),
    (192, 384, 2, 1, True),
    (384, 256, 1, 2, True),
    (256, 2, 1, 4, False),
)


def param_count(layers=LAYERS) -> int:
    return sum(9 * ic * oc + oc for ic, oc, _, _, _ in layers)


def unpack(params, layers=LAYERS):
    """Flat parameter vector -> list of (W [OC,3,3,IC], b [OC])."""
    out, o = [], 0
    for ic, oc, _, _, _ in layers:
        w = np.asarray(params[o:o + 9 * ic * oc], dtype=np.float64).reshape(oc, 3, 3, ic)
        o += 9 * ic * oc
        b = np.asarray(params[o:o + oc], dtype=np.float64)
        o += oc
        out.append((w, b))
    return out


def pack(wb):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in wb])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 is the upper 16 bits of an IEEE binary32: round the binary32 value at bit 16 by adding
    0x7FFF plus the lowest kept bit, then clear the low half."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def upsample(x, f):
    """Nearest-neighbour upsampling of [B, H, W, C] by an integer factor."""
    if f == 1:
        return x
    return np.repeat(np.repeat(x, f, axis=1), f, axis=2)


def block_sum(x, f):
    """Adjoint of `upsample`: sum of every f x f block."""
    if f == 1:
        return x
    B, H, W, C = x.shape
    return x.reshape(B, H // f, f, W // f, f, C).sum(axis=(2, 4))


def conv_forward(x, w, b, stride, up):
    """z[b, oy, ox, o] = b[o] + sum_{ky, kx, c} w[o, ky, kx, c] u[b, s oy + ky - 1, s ox + kx - 1, c],
    u = upsample(x, up) with zeros outside."""
    u = upsample(x, up)
    B, H, W, C = u.shape
    OH, OW = (H + stride - 1) // stride, (W + stride - 1) // stride
    up_ = np.zeros((B, H + 2, W + 2, C))
    up_[:, 1:H + 1, 1:W + 1, :] = u
    z = np.zeros((B, OH, OW, w.shape[0])) + b
    for ky in range(3):
        for kx in range(3):
            tap = up_[:, ky:ky + stride * (OH - 1) + 1:stride, kx:kx + stride * (OW - 1) + 1:stride, :]
            z += tap @ w[:, ky, kx, :].T
    return z


def conv_backward(x, w, stride, up, dz):
    """Gradients of sum(dz * conv_forward(x, w, b)) with respect to x, w and b."""
    u = upsample(x, up)
    B, H, W, C = u.shape
    OH, OW = dz.shape[1], dz.shape[2]
    up_ = np.zeros((B, H + 2, W + 2, C))
    up_[:, 1:H + 1, 1:W + 1, :] = u
    du_ = np.zeros_like(up_)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            sl = (slice(None), slice(ky, ky + stride * (OH - 1) + 1, stride),
                  slice(kx, kx + stride * (OW - 1) + 1, stride), slice(None))
            dw[:, ky, kx, :] = np.tensordot(dz, up_[sl], axes=([0, 1, 2], [0, 1, 2]))
            du_[sl] += dz @ w[:, ky, kx, :]
    db = dz.sum(axis=(0, 1, 2))
    dx = block_sum(du_[:, 1:H + 1, 1:W + 1, :], up)
    return dx, dw, db


def net_input(I, s_in, bf=True):
    x = s_in * np.log1p(np.asarray(I, dtype=np.float64))[..., None]
    return bf16(x) if bf else x


def forward(params, I, s_in, bf=True, layers=LAYERS):
    """Network output [B, H/2, W/2, 2] and the stored activations (inputs of every layer)."""
    wb = unpack(params, layers)
    a = net_input(I, s_in, bf)
    acts = [a]
    for li, ((w, b), (_, _, stride, up, relu)) in enumerate(zip(wb, layers)):
        z = conv_forward(a, bf16(w) if bf else w, b, stride, up)
        if relu:
            a = np.maximum(z, 0.0)
            a = bf16(a) if bf else a
            acts.append(a)
        else:
            return z, acts
    raise ValueError("the last layer must be linear")


def loss_and_grad(params, I, Y, s_in, bf=True, layers=LAYERS):
    """MSE loss of the batch and its gradient with respect to the flat parameter vector."""
    out, acts = forward(params, I, s_in, bf, layers)
    wb = unpack(params, layers)
    Y = np.asarray(Y, dtype=np.float64)
    n = out.size
    loss = float(np.mean((out - Y) ** 2))
    dz = 2.0 * (out - Y) / n
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        _, _, stride, up, _ = layers[li]
        dz = bf16(dz) if bf else dz
        w = bf16(wb[li][0]) if bf else wb[li][0]
        dx, dw, db = conv_backward(acts[li], w, stride, up, dz)
        grads[li] = (dw, db)
        if li > 0:
            dz = dx * (acts[li] > 0)  # ReLU of the layer below (its stored output)
    return loss, pack(grads)


def targets(amp, phase, corners, N):
    """Training targets: the central N/2 x N/2 of each N x N window at integer corner (i0, i1) of
    the depth-summed phase and log-amplitude, [B, N/2, N/2, 2]."""
    phi = np.asarray(phase, dtype=np.float64).sum(axis=0)
    la = np.log(np.asarray(amp, dtype=np.float64)).sum(axis=0)
    h = N // 2
    q = N // 4
    out = np.zeros((len(corners), h, h, 2))
    for k, (i0, i1) in enumerate(corners):
        out[k, :, :, 0] = phi[i0 + q:i0 + q + h, i1 + q:i1 + q + h]
        out[k, :, :, 1] = la[i0 + q:i0 + q + h, i1 + q:i1 + q + h]
    return out


def stitch(pred, corners, weight, H, W, N, Nz):
    """Initial object from predicted patches: the weight-averaged depth sums, split evenly over
    Nz slices (phase / Nz, amplitude exp(log-amplitude / Nz)); uncovered pixels stay flat."""
    h, q = N // 2, N // 4
    num = np.zeros((H, W, 2))
    den = np.zeros((H, W))
    for k, (i0, i1) in enumerate(corners):
        num[i0 + q:i0 + q + h, i1 + q:i1 + q + h, :] += weight[..., None] * pred[k]
        den[i0 + q:i0 + q + h, i1 + q:i1 + q + h] += weight
    mean = np.where(den[..., None] > 0, num / np.where(den > 0, den, 1.0)[..., None], 0.0)
    phase = np.repeat((mean[..., 0] / Nz)[None], Nz, axis=0)
    amp = np.repeat(np.exp(mean[..., 1] / Nz)[None], Nz, axis=0)
    return amp, phase


def nmse(phi_hat, phi, roi):
    """sum_roi (phi_hat - phi - c)^2 / sum_roi (phi - mean phi)^2 with c = mean_roi(phi_hat - phi)
    (removes the global phase offset); phi are depth-summed phases, roi = (r0, r1, c0, c1)."""
    r0, r1, c0, c1 = roi
    a = np.asarray(phi_hat, dtype=np.float64)[r0:r1, c0:c1]
    b = np.asarray(phi, dtype=np.float64)[r0:r1, c0:c1]
    d = a - b
    d = d - d.mean()
    e = b - b.mean()
    return float((d * d).sum() / (e * e).sum())
