"""Python binding of the learned initialiser (include/pty_cnn.h): argument marshalling only, every
step runs in the library's kernels.

    net = Cnn(S=128, max_batch=256)             # parameters from a seeded He initialisation
    net.train_step(I, Y, lr=1e-3)               # I [B,S,S] patterns, Y [B,S/2,S/2,2] targets
    pred = net.predict(I)                       # [B,S/2,S/2,2]: depth-summed phase, log-amplitude
    st = Stitcher(S, Nz, H, W, weight); st.add(pred, pos, idx); amp, phase = st.finish()
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

# layer table of the network (in, out channels) in parameter order; see include/pty_cnn.h
LAYER_CHANNELS = ((1, 48), (48, 96), (96, 192), (192, 384), (384, 256), (256, 2))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def he_init(seed: int) -> np.ndarray:
    """Seeded He-normal weights (std sqrt(2 / fan_in)), zero biases, in the flat parameter layout;
    the output layer is scaled by 0.1 so that the untrained network predicts near zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for k, (ic, oc) in enumerate(LAYER_CHANNELS):
        w = rng.standard_normal((oc, 3, 3, ic)) * np.sqrt(2.0 / (9 * ic))
        if k == len(LAYER_CHANNELS) - 1:
            w *= 0.1
        parts += [w.ravel(), np.zeros(oc)]
    return np.concatenate(parts).astype(np.float32)


class Cnn:
    """Network parameters (FP32 master copy), Adam state and a workspace for batches of up to
    max_batch patterns of S x S on one device."""

    def __init__(self, S: int = 128, max_batch: int = 256, seed: int = 2000, device="cuda", s_in: float = 0.2,
                 params: torch.Tensor | None = None):
        self.S, self.max_batch, self.s_in = S, max_batch, float(s_in)
        self.device = torch.device(device)
        n = _lib.pty_cnn_param_count()
        if params is None:
            params = torch.tensor(he_init(seed), device=self.device)
        assert params.numel() == n and params.dtype == torch.float32
        self.params = params.contiguous()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.step_count = 0
        self.ws_bytes = _lib.pty_cnn_workspace_size(S, max_batch)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)

    def _batch(self, I):
        B = I.shape[0]
        if B > self.max_batch:
            raise ValueError("batch %d > max_batch %d" % (B, self.max_batch))
        assert I.dtype == torch.float32 and I.is_contiguous() and tuple(I.shape[1:]) == (self.S, self.S)
        return B

    def predict(self, I: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        B = self._batch(I)
        h = self.S // 2
        if out is None:
            out = torch.empty((B, h, h, 2), dtype=torch.float32, device=self.device)
        _lib.pty_cnn_forward(self.S, B, _ptr(self.params), _ptr(I), self.s_in, _ptr(out), _ptr(self.ws),
                             self.ws_bytes, _stream(self.device))
        return out

    def loss_grad(self, I: torch.Tensor, Y: torch.Tensor, pred: torch.Tensor | None = None):
        """(loss [1] float64 device tensor, gradient of the flat parameters) for one batch."""
        B = self._batch(I)
        assert Y.dtype == torch.float32 and Y.is_contiguous() and Y.shape[0] == B
        _lib.pty_cnn_loss_grad(self.S, B, _ptr(self.params), _ptr(I), _ptr(Y), self.s_in, _ptr(self.loss),
                               _ptr(self.grad), _ptr(pred), _ptr(self.ws), self.ws_bytes, _stream(self.device))
        return self.loss, self.grad

    def state(self, B: int, layer: int, what: str = "act") -> torch.Tensor:
        """FP32 copy of layer `layer`'s stored activation ("act", layers 1..5) or of the gradient
        dL/dz that fed its weight and input gradients ("dz", layers 1..6), as left by the last
        predict / loss_grad call with batch B."""
        h = self.S // 2 ** layer if layer <= 4 else (self.S // 8 if layer == 5 else self.S // 2)
        C = LAYER_CHANNELS[layer - 1][1]
        out = torch.empty((B, h, h, C), dtype=torch.float32, device=self.device)
        _lib.pty_cnn_read_state(self.S, B, _ptr(self.ws), self.ws_bytes, layer, 0 if what == "act" else 1, _ptr(out),
                                _stream(self.device))
        return out

    def train_step(self, I: torch.Tensor, Y: torch.Tensor, lr: float = 1e-3) -> torch.Tensor:
        B = self._batch(I)
        assert Y.dtype == torch.float32 and Y.is_contiguous() and Y.shape[0] == B
        self.step_count += 1
        _lib.pty_cnn_train_step(self.S, B, _ptr(self.params), _ptr(self.m), _ptr(self.v), _ptr(self.grad),
                                self.step_count, lr, _ptr(I), _ptr(Y), self.s_in, _ptr(self.loss), _ptr(self.ws),
                                self.ws_bytes, _stream(self.device))
        return self.loss


def targets(S: int, amp: torch.Tensor, phase: torch.Tensor, pos: torch.Tensor, idx: torch.Tensor,
            out: torch.Tensor | None = None) -> torch.Tensor:
    """Central (S/2)^2 of each probe window of the depth-summed phase and log-amplitude."""
    Nz, H, W = amp.shape
    B = idx.numel()
    if out is None:
        out = torch.empty((B, S // 2, S // 2, 2), dtype=torch.float32, device=amp.device)
    _lib.pty_cnn_targets(S, Nz, H, W, _ptr(amp), _ptr(phase), _ptr(pos), _ptr(idx), B, _ptr(out), _stream(amp.device))
    return out


class Stitcher:
    """Accumulates predicted patches into an object of [H, W] and turns them into amp/phase [Nz, H, W]."""

    def __init__(self, S: int, Nz: int, H: int, W: int, weight: torch.Tensor, device="cuda"):
        self.S, self.Nz, self.H, self.W = S, Nz, H, W
        self.device = torch.device(device)
        self.weight = weight.to(device=self.device, dtype=torch.float32).contiguous()
        assert tuple(self.weight.shape) == (S // 2, S // 2)
        self.num = torch.zeros((H, W, 2), dtype=torch.float32, device=self.device)
        self.den = torch.zeros((H, W), dtype=torch.float32, device=self.device)

    def add(self, pred: torch.Tensor, pos: torch.Tensor, idx: torch.Tensor):
        _lib.pty_cnn_stitch(self.S, self.H, self.W, _ptr(pred), _ptr(pos), _ptr(idx), idx.numel(), _ptr(self.weight),
                            _ptr(self.num), _ptr(self.den), _stream(self.device))

    def finish(self, amp: torch.Tensor | None = None, phase: torch.Tensor | None = None):
        shape = (self.Nz, self.H, self.W)
        if amp is None:
            amp = torch.empty(shape, dtype=torch.float32, device=self.device)
        if phase is None:
            phase = torch.empty(shape, dtype=torch.float32, device=self.device)
        _lib.pty_cnn_stitch_finish(self.Nz, self.H, self.W, _ptr(self.num), _ptr(self.den), _ptr(amp), _ptr(phase),
                                   _stream(self.device))
        return amp, phase
