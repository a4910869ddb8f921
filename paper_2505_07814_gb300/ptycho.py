"""PyTorch-facing wrapper of the C ABI: tensors in, device pointers out, nothing computed here.

PyTorch supplies device memory and the current stream; every step of the model runs in the CUDA
kernels of libpty.so.  If the library is missing, constructing `Ptycho` raises.
"""
from __future__ import annotations

import dataclasses

import torch

from . import _lib

LOSS = {"poisson": _lib.PTY_LOSS_POISSON, "gaussian": _lib.PTY_LOSS_GAUSSIAN}
FFT_IMPL = {"fp32": _lib.PTY_FFT_FP32, "bf16": _lib.PTY_FFT_SPLIT_BF16, "fp16": _lib.PTY_FFT_SPLIT_FP16,
            "bf16x3": _lib.PTY_FFT_SPLIT3_BF16}
GRAD_BITS = {"amp": _lib.PTY_GRAD_AMP, "phase": _lib.PTY_GRAD_PHASE, "probe": _lib.PTY_GRAD_PROBE,
             "pos": _lib.PTY_GRAD_POS, "tilt": _lib.PTY_GRAD_TILT, "dz": _lib.PTY_GRAD_DZ}


@dataclasses.dataclass
class Geometry:
    N: int
    M: int
    Nz: int
    H: int
    W: int
    Ntot: int
    dx: float
    lam: float
    loss: str = "poisson"
    p: float = 0.0  # <= 0: default exponent (1 Poisson, 0.5 Gaussian)
    eps: float = 1e-6
    grads: tuple = ("amp", "phase", "probe", "pos", "tilt", "dz")
    global_tilt: bool = False
    ckpt_stride: int = 1  # 1: checkpoint every slice; K > 1: re-run K-slice segments in the adjoint
    # per-slice DFTs: "fp32" shared-memory FFT; split-precision tensor-core GEMMs "bf16" / "fp16"
    # (hi + lo pieces, three products) or "bf16x3" (three bf16 pieces, six products)
    fft: str = "fp32"
    # extra loss terms (Eq. 7-9): PACBED and phase sparsity, weight 0 = off, exponent <= 0 = default
    w_pacbed: float = 0.0
    p_pacbed: float = 0.0
    w_sparse: float = 0.0
    p_sparse: float = 0.0
    obj_modes: int = 1  # object modes K (Eq. 2): amp / phase are [K, Nz, H, W] when K > 1

    @property
    def nobj(self) -> int:
        """Elements of the amplitude (or phase) array: K x Nz x H x W."""
        return max(self.obj_modes, 1) * self.Nz * self.H * self.W

    @property
    def grad_mask(self) -> int:
        m = 0
        for g in self.grads:
            m |= GRAD_BITS[g]
        return m

    def c(self) -> _lib.pty_geom:
        return _lib.pty_geom(self.N, self.M, self.Nz, self.H, self.W, self.Ntot, self.dx, self.lam,
                             LOSS[self.loss], self.p, self.eps, self.grad_mask, int(self.global_tilt),
                             int(self.ckpt_stride), FFT_IMPL[self.fft], float(self.w_pacbed), float(self.p_pacbed),
                             float(self.w_sparse), float(self.p_sparse), int(self.obj_modes))

    def checkpoint_bytes(self, B: int) -> int:
        """Bytes the adjoint's forward record takes for a batch of B positions (see ckpt_stride)."""
        wave = 8 * self.N * self.N * B * self.M * max(self.obj_modes, 1)
        if self.ckpt_stride <= 1 or self.fft != "fp32":
            return wave * (2 * self.Nz - 1)
        K = min(self.ckpt_stride, self.Nz)
        return wave * ((self.Nz + K - 1) // K - 1 + 2 * K + 1)


@dataclasses.dataclass
class Params:
    """Device tensors: amp/phase float32 [Nz,H,W] (or [K,Nz,H,W] with object modes), probe complex64 [M,N,N], pos float32 [Ntot,2],
    tilt float32 [Ntot,2] (or [2]), dz float32 [1]."""
    amp: torch.Tensor
    phase: torch.Tensor
    probe: torch.Tensor
    pos: torch.Tensor
    tilt: torch.Tensor
    dz: torch.Tensor

    @staticmethod
    def from_numpy(w, device="cuda", global_tilt=False) -> "Params":
        f32 = dict(dtype=torch.float32, device=device)
        tilt = w.tilt[0] if global_tilt else w.tilt
        return Params(amp=torch.tensor(w.amp, **f32), phase=torch.tensor(w.phase, **f32),
                      probe=torch.tensor(w.probe, dtype=torch.complex64, device=device),
                      pos=torch.tensor(w.pos, **f32), tilt=torch.tensor(tilt, **f32),
                      dz=torch.tensor([w.dz], **f32))

    def zeros_like(self) -> "Params":
        return Params(*(torch.zeros_like(t) for t in dataclasses.astuple(self)))


def _ptr(t, dtype=None, numel=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, has %d" % (name, numel, t.numel()))
    return t.data_ptr()


class Ptycho:
    """One reconstruction problem on one device, with a workspace sized for batches up to max_batch.

    ckpt_budget (bytes): let the library choose the adjoint's memory plan (pty_plan_ckpt): keep
    every slice's forward waves when the workspace fits the budget, else the recompute stride of
    least work that does; geom.ckpt_stride is then replaced and the plan is in `self.plan`."""

    def __init__(self, geom: Geometry, max_batch: int, device="cuda", ckpt_budget: int | None = None):
        _lib.load()
        self.plan = None
        if ckpt_budget is not None:
            stride, need = _lib.pty_plan_ckpt(geom.c(), max_batch, int(ckpt_budget))
            geom = dataclasses.replace(geom, ckpt_stride=stride)
            self.plan = {"ckpt_stride": stride, "workspace_bytes": need, "budget_bytes": int(ckpt_budget)}
        self.geom = geom
        self.cg = geom.c()
        self.device = torch.device(device)
        self.max_batch = max_batch
        self.ws_bytes = _lib.pty_workspace_size(self.cg, max_batch)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        self._generation = 0  # bumped by every forward_save (one saved forward per workspace)
        self._saved = None

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def _param_ptrs(self, p: Params):
        g = self.geom
        nobj = g.nobj
        ntilt = 2 if g.global_tilt else 2 * g.Ntot
        return (_ptr(p.amp, torch.float32, nobj, "amp"), _ptr(p.phase, torch.float32, nobj, "phase"),
                _ptr(p.probe, torch.complex64, g.M * g.N * g.N, "probe"),
                _ptr(p.pos, torch.float32, 2 * g.Ntot, "pos"), _ptr(p.tilt, torch.float32, ntilt, "tilt"),
                _ptr(p.dz, torch.float32, 1, "dz"))

    def _idx(self, idx):
        idx = torch.as_tensor(idx, dtype=torch.int32, device=self.device).contiguous()
        if idx.numel() > self.max_batch:
            raise ValueError("batch of %d exceeds max_batch %d" % (idx.numel(), self.max_batch))
        return idx

    def forward(self, params: Params, idx, out: torch.Tensor | None = None) -> torch.Tensor:
        """Modelled patterns I[b] for scan positions idx (Eq. 1-4), float32 [B,N,N], DC-centred."""
        idx = self._idx(idx)
        B, N = idx.numel(), self.geom.N
        if out is None:
            out = torch.empty((B, N, N), dtype=torch.float32, device=self.device)
        _lib.pty_forward(self.cg, B, _ptr(idx), *self._param_ptrs(params),
                         _ptr(out, torch.float32, B * N * N, "I_model"), self.ws.data_ptr(), self.ws_bytes,
                         self._stream())
        return out

    def loss_grad(self, params: Params, idx, I_meas: torch.Tensor, grads: Params | None = None,
                  accumulate: bool = False, I_model: torch.Tensor | None = None,
                  whole_stats: torch.Tensor | None = None):
        """Loss (Eq. 5/6) of the batch and gradients of every parameter named in geom.grads.

        whole_stats: when idx is one part of a larger batch (a data-parallel rank's share, or a
        sub-batch of an accumulated gradient), the float64 [3] device tensor of the whole batch's
        loss statistics (the sum of every part's `loss_stats`); the loss and gradients are then this
        part's share of the whole batch's (pty_loss_grad_part).
        Returns (loss as a float64 device tensor of one element, grads)."""
        idx = self._idx(idx)
        g = self.geom
        B = idx.numel()
        if grads is None:
            grads = params.zeros_like()
        gp = self._param_ptrs(grads)
        args = (_ptr(idx), *self._param_ptrs(params), _ptr(I_meas, torch.float32, g.Ntot * g.N * g.N, "I_meas"))
        tail = (self.loss.data_ptr(), _ptr(I_model, torch.float32, B * g.N * g.N, "I_model"), *gp, int(accumulate),
                self.ws.data_ptr(), self.ws_bytes, self._stream())
        if whole_stats is None:
            _lib.pty_loss_grad(self.cg, B, *args, *tail)
        else:
            _lib.pty_loss_grad_part(self.cg, B, *args, _ptr(whole_stats, torch.float64, 3, "whole_stats"), *tail)
        return self.loss, grads

    def loss_stats(self, params: Params, idx, I_meas: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """This batch's loss statistics {sum I_meas^p, sum of squared residuals (Gaussian), pixels x
        patterns} as a float64 [3] device tensor (pty_loss_stats).  The sum over the parts of a
        batch is the `whole_stats` argument of loss_grad."""
        idx = self._idx(idx)
        g = self.geom
        if out is None:
            out = torch.empty(3, dtype=torch.float64, device=self.device)
        _lib.pty_loss_stats(self.cg, idx.numel(), _ptr(idx), *self._param_ptrs(params),
                            _ptr(I_meas, torch.float32, g.Ntot * g.N * g.N, "I_meas"),
                            _ptr(out, torch.float64, 3, "stats"), self.ws.data_ptr(), self.ws_bytes,
                            self._stream())
        return out

    def forward_save(self, params: Params, idx, out: torch.Tensor | None = None) -> torch.Tensor:
        """Modelled patterns, keeping in the workspace what `backward` needs (pty_forward_save)."""
        idx = self._idx(idx)
        B, N = idx.numel(), self.geom.N
        if out is None:
            out = torch.empty((B, N, N), dtype=torch.float32, device=self.device)
        self._generation += 1
        _lib.pty_forward_save(self.cg, B, _ptr(idx), *self._param_ptrs(params),
                              _ptr(out, torch.float32, B * N * N, "I_model"), self.ws.data_ptr(), self.ws_bytes,
                              self._stream())
        self._saved = (idx, self._generation)
        return out

    def backward(self, params: Params, idx, dL_dI: torch.Tensor, grads: Params | None = None,
                 accumulate: bool = False) -> Params:
        """Gradients for dL/dI [B,N,N] (DC-centred) through the forward of the last `forward_save`."""
        idx = self._idx(idx)
        B, N = idx.numel(), self.geom.N
        if grads is None:
            grads = params.zeros_like()
        _lib.pty_backward(self.cg, B, _ptr(idx), *self._param_ptrs(params),
                          _ptr(dL_dI.contiguous(), torch.float32, B * N * N, "dL_dI"), *self._param_ptrs(grads),
                          int(accumulate), self.ws.data_ptr(), self.ws_bytes, self._stream())
        return grads

    def status(self) -> int:
        """Device status bits of the last call (synchronises the current stream)."""
        return _lib.pty_status(self.ws.data_ptr(), self._stream())


class Adam:
    """Adam state (PyTorch semantics) for pty_step / pty_adam_update, one learning rate per parameter.
    A learning rate of 0 (or a parameter missing from geom.grads) freezes that parameter."""

    def __init__(self, params: Params, lr: dict, betas=(0.9, 0.999), eps=1e-8):
        self.m = params.zeros_like()
        self.v = params.zeros_like()
        self.lr = {k: float(lr.get(k, 0.0)) for k in GRAD_BITS}
        self.betas, self.eps = betas, eps
        self.t = 0

    def c(self) -> _lib.pty_adam:
        a = _lib.pty_adam()
        for name in GRAD_BITS:
            setattr(a, "m_" + name, getattr(self.m, name).data_ptr())
            setattr(a, "v_" + name, getattr(self.v, name).data_ptr())
            setattr(a, "lr_" + name, self.lr[name])
        a.beta1, a.beta2 = self.betas
        a.eps = self.eps
        return a


def step(pt: Ptycho, params: Params, grads: Params, adam: Adam, idx, I_meas: torch.Tensor):
    """One Adam iteration on one batch through pty_step; returns the batch loss (device tensor)."""
    idx = pt._idx(idx)
    g = pt.geom
    adam.t += 1
    _lib.pty_step(pt.cg, idx.numel(), _ptr(idx), *pt._param_ptrs(params),
                  _ptr(I_meas, torch.float32, g.Ntot * g.N * g.N, "I_meas"), pt.loss.data_ptr(),
                  *pt._param_ptrs(grads), adam.c(), adam.t, pt.ws.data_ptr(), pt.ws_bytes, pt._stream())
    return pt.loss


def constrain(pt: Ptycho, params: Params, phase_positivity: float = 0.0, rz_sigma: float = 0.0,
              rz_relax: float = 1.0, kz_beta: float = 0.0, kz_alpha: float = 0.0, kz_relax: float = 0.0,
              orthogonalize_probe: bool = False):
    """Constraints after an optimiser step (pty_constrain), in place on params: probe-mode
    orthogonalisation; then on amp / phase the relaxed k_z filter (Eq. 10-12), the relaxed depth
    blur along the slices (Eq. 13) and the relaxed phase >= 0 clip."""
    g = pt.geom
    nobj = g.nobj
    c = _lib.pty_constraints(float(phase_positivity), float(rz_sigma), float(rz_relax), float(kz_beta),
                             float(kz_alpha), float(kz_relax), int(bool(orthogonalize_probe)))
    need = _lib.pty_constrain_workspace_size(pt.cg, c)
    ws = getattr(pt, "_constrain_ws", None)
    if need and (ws is None or ws.numel() < need):
        ws = torch.empty(need, dtype=torch.uint8, device=pt.device)
        pt._constrain_ws = ws
    _lib.pty_constrain(pt.cg, _ptr(params.amp, torch.float32, nobj, "amp"),
                       _ptr(params.phase, torch.float32, nobj, "phase"),
                       _ptr(params.probe, torch.complex64, g.M * g.N * g.N, "probe"),
                       _ptr(params.dz, torch.float32, 1, "dz"), c, ws.data_ptr() if need else None, need,
                       pt._stream())


class _ForwardModel(torch.autograd.Function):
    """I = f(amp, phase, probe, pos, tilt, dz) for one batch, differentiated by the library's adjoint."""

    @staticmethod
    def forward(ctx, pt, idx, amp, phase, probe, pos, tilt, dz):
        params = Params(amp.detach(), phase.detach(), probe.detach(), pos.detach(), tilt.detach(), dz.detach())
        I = pt.forward_save(params, idx)
        ctx.pt, ctx.idx, ctx.gen = pt, idx, pt._generation
        ctx.params = params
        return I

    @staticmethod
    def backward(ctx, gI):
        pt = ctx.pt
        if pt._generation != ctx.gen:
            raise RuntimeError("another forward ran on this Ptycho workspace before backward; one forward "
                               "per workspace may be differentiated at a time")
        g = pt.backward(ctx.params, ctx.idx, gI.to(torch.float32))
        want = set(pt.geom.grads)
        out = [g.amp, g.phase, g.probe, g.pos, g.tilt, g.dz]
        out = [t if n in want else None for n, t in zip(("amp", "phase", "probe", "pos", "tilt", "dz"), out)]
        return (None, None, *out)


def forward_model(pt: Ptycho, params: Params, idx) -> torch.Tensor:
    """Differentiable modelled patterns [B,N,N] (DC-centred) for scan positions idx.

    The backward pass runs the library's hand-written adjoint (pty_backward) with the checkpoint /
    recompute plan of pt.geom.ckpt_stride; gradients flow to every tensor in `params` named in
    pt.geom.grads.  One forward per Ptycho workspace may be differentiated at a time."""
    return _ForwardModel.apply(pt, pt._idx(idx), params.amp, params.phase, params.probe, params.pos,
                               params.tilt, params.dz)
