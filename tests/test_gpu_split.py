"""Split-precision DFT-GEMM path (pty_geom.fft_impl) against the FP64 oracle.

Every per-slice 2D DFT runs as dense DFT matrix products on the tensor cores with each FP32
operand cut into 16-bit pieces and FP32 accumulation.  The bars are relative L2 <= 1e-4 on
intensities and loss and <= 1e-3 on gradients.  fp16 hi + lo keeps 22 significant bits and bf16 with
three pieces 24: both meet them.  bf16 hi + lo keeps 16 bits, 2^8 fewer than FP32, so its transforms
carry about 2^8 times the FP32 path's rounding error: it meets the intensity bar but its gradients
miss 1e-3 (about 1.8e-3 on the multislice cases).  Those cases are reported as expected failures
with the measured error, after the intensity bar has been checked.
"""
import numpy as np
import pytest

from oracle import ptycho as O
from tests.cases import make_case, oracle_grads, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_I = 1e-4
TOL_G = {"fp16": 1e-3, "bf16x3": 1e-3, "bf16": 1e-3}
FORMATS = ["bf16", "fp16", "bf16x3"]
GRADS = ("amp", "phase", "probe", "pos", "tilt", "dz")


def _gpu(case, fft, grads=GRADS, ckpt_stride=1):
    from paper_2505_07814_gb300.ptycho import Geometry, Params, Ptycho
    g = case.geom
    geom = Geometry(N=g.N, M=g.M, Nz=g.Nz, H=g.H, W=g.W, Ntot=case.Ntot, dx=g.dx, lam=g.lam, loss=g.loss,
                    eps=g.eps, grads=tuple(grads), global_tilt=g.global_tilt, ckpt_stride=ckpt_stride, fft=fft)
    dev = torch.device("cuda")
    f32 = dict(dtype=torch.float32, device=dev)
    params = Params(amp=torch.tensor(case.amp, **f32), phase=torch.tensor(case.phase, **f32),
                    probe=torch.tensor(case.probe, dtype=torch.complex64, device=dev),
                    pos=torch.tensor(case.pos, **f32), tilt=torch.tensor(case.tilt, **f32),
                    dz=torch.tensor([case.dz], **f32))
    return Ptycho(geom, case.Ntot, device=dev), params, torch.tensor(case.I_meas, **f32)


def _np(t):
    return t.detach().cpu().numpy()


def _errors(case, idx, fft, grads=GRADS, ckpt_stride=1):
    pt, params, I_meas = _gpu(case, fft, grads, ckpt_stride)
    I_model = torch.empty((len(idx), case.geom.N, case.geom.N), dtype=torch.float32, device="cuda")
    loss, g = pt.loss_grad(params, idx, I_meas, I_model=I_model)
    torch.cuda.synchronize()
    assert pt.status() == 0
    ref = oracle_grads(case, idx)
    err = {"I": rel_l2(_np(I_model), ref.I_model), "loss": abs(loss.item() - ref.loss) / abs(ref.loss)}
    for name in grads:
        got = _np(getattr(g, name))
        err[name] = rel_l2(got[0] if name == "dz" else got, getattr(ref, name))
    I_fwd = pt.forward(params, idx)
    torch.cuda.synchronize()
    err["I_fwd"] = rel_l2(_np(I_fwd), ref.I_model)
    return err


def _assert(err, fft):
    for k in ("I", "loss", "I_fwd"):
        assert err[k] <= TOL_I, (k, err[k], err)
    miss = {k: v for k, v in err.items() if k not in ("I", "loss", "I_fwd") and v > TOL_G[fft]}
    if miss and fft == "bf16":
        pytest.xfail("bf16 hi + lo gradients miss the 1e-3 bar: %s" % ", ".join("%s %.2e" % kv for kv in miss.items()))
    assert not miss, (miss, err)


@pytest.mark.parametrize("fft", FORMATS)
@pytest.mark.parametrize("loss", [O.POISSON, O.GAUSSIAN])
def test_split_multislice_multimode_n64(fft, loss):
    case = make_case(N=64, M=3, Nz=4, scan=(3, 4), loss=loss, seed=11)
    _assert(_errors(case, list(range(case.Ntot)), fft), fft)


@pytest.mark.parametrize("fft", FORMATS)
def test_split_multislice_n128_ragged(fft):
    # 11 of 12 positions: B*M*N = 11*2*128 rows, a ragged last GEMM row tile
    case = make_case(N=128, M=2, Nz=3, scan=(3, 4), seed=12, step=9, pad=(5, 9))
    idx = [0, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11]
    _assert(_errors(case, idx, fft), fft)


@pytest.mark.parametrize("fft", FORMATS)
def test_split_single_slice_global_tilt(fft):
    case = make_case(N=64, M=1, Nz=1, scan=(2, 3), global_tilt=True, seed=13)
    _assert(_errors(case, list(range(case.Ntot)), fft), fft)


def test_split_ignores_ckpt_stride_and_matches_fp32_path():
    """ckpt_stride > 1 does not change the split modes; the two precisions agree with the FP32 FFT
    path to well inside their own tolerance."""
    case = make_case(N=64, M=2, Nz=5, scan=(3, 3), seed=14)
    idx = list(range(case.Ntot))
    out = {}
    for fft, K in (("fp32", 1), ("bf16", 1), ("bf16", 3), ("fp16", 1), ("bf16x3", 1)):
        pt, params, I_meas = _gpu(case, fft, ckpt_stride=K)
        loss, g = pt.loss_grad(params, idx, I_meas)
        torch.cuda.synchronize()
        assert pt.status() == 0
        out[(fft, K)] = (loss.item(), _np(g.amp), _np(g.probe))
    l1, a1, p1 = out[("bf16", 1)]
    l3, a3, p3 = out[("bf16", 3)]
    assert l1 == l3 and rel_l2(a3, a1) < 1e-6
    lf, af, pf = out[("fp32", 1)]
    miss = {}
    for key in (("fp16", 1), ("bf16x3", 1), ("bf16", 1)):
        ls, as_, ps = out[key]
        assert abs(ls - lf) <= TOL_I * abs(lf)
        for name, e in (("amp", rel_l2(as_, af)), ("probe", rel_l2(ps, pf))):
            if e > TOL_G[key[0]]:
                miss["%s %s" % (key[0], name)] = e
    if miss and all(k.startswith("bf16 ") for k in miss):
        pytest.xfail("bf16 hi + lo gradients miss the 1e-3 bar: %s" % ", ".join("%s %.2e" % kv for kv in miss.items()))
    assert not miss, miss


def _torch_poisson(I, I_meas_b, eps=1e-6):
    I = I.to(torch.float64)
    d = I_meas_b.to(torch.float64)
    return -torch.mean(d * torch.log(I + eps) - I) / torch.mean(d)


@pytest.mark.parametrize("fft", FORMATS)
def test_split_autograd_backward(fft):
    """forward_save + backward (the torch.autograd path) under a Poisson loss written in torch."""
    from paper_2505_07814_gb300.ptycho import Params, forward_model
    case = make_case(N=64, M=2, Nz=3, scan=(2, 3), seed=15)
    idx = [4, 0, 2, 5]
    pt, params, I_meas = _gpu(case, fft)
    leaves = {n: getattr(params, n).clone().requires_grad_(True) for n in GRADS}
    I = forward_model(pt, Params(**leaves), idx)
    loss = _torch_poisson(I, I_meas[torch.tensor(idx, device="cuda")])
    loss.backward()
    torch.cuda.synchronize()
    ref = oracle_grads(case, idx)
    assert rel_l2(_np(I), ref.I_model) <= TOL_I
    assert abs(loss.item() - ref.loss) <= TOL_I * abs(ref.loss)
    err = {"I": 0.0, "loss": 0.0, "I_fwd": 0.0}
    for name in GRADS:
        got = _np(leaves[name].grad)
        err[name] = rel_l2(got[0] if name == "dz" else got, getattr(ref, name))
    _assert(err, fft)
