"""The PACBED and phase-sparsity terms of the total loss (Eq. 7-9) on the GPU against the oracle:
loss and every gradient, through the FP32 FFT path (shared-memory and cluster loss kernels) and
the split-precision GEMM path."""
import dataclasses

import numpy as np
import pytest

from oracle import ptycho as O
from tests.cases import make_case, oracle_grads, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ("amp", "phase", "probe", "pos", "tilt", "dz")


def _run(case, idx, terms, fft="fp32", grads=NAMES):
    from paper_2505_07814_gb300.ptycho import Geometry, Params, Ptycho
    g = case.geom
    geom = Geometry(N=g.N, M=g.M, Nz=g.Nz, H=g.H, W=g.W, Ntot=case.Ntot, dx=g.dx, lam=g.lam, loss=g.loss,
                    eps=g.eps, grads=tuple(grads), global_tilt=g.global_tilt, fft=fft, **terms)
    f = dict(dtype=torch.float32, device="cuda")
    params = Params(amp=torch.tensor(case.amp, **f), phase=torch.tensor(case.phase, **f),
                    probe=torch.tensor(case.probe, dtype=torch.complex64, device="cuda"),
                    pos=torch.tensor(case.pos, **f), tilt=torch.tensor(case.tilt, **f),
                    dz=torch.tensor([case.dz], **f))
    pt = Ptycho(geom, case.Ntot)
    loss, gr = pt.loss_grad(params, idx, torch.tensor(case.I_meas, **f))
    torch.cuda.synchronize()
    assert pt.status() == 0
    return loss.item(), gr


def _oracle(case, idx, terms):
    c = dataclasses.replace(case, geom=dataclasses.replace(case.geom, w_pacbed=terms.get("w_pacbed", 0.0),
                                                           p_pacbed=terms.get("p_pacbed") or None,
                                                           w_sparse=terms.get("w_sparse", 0.0),
                                                           p_sparse=terms.get("p_sparse") or None))
    return oracle_grads(c, idx)


@pytest.mark.parametrize("N,M,Nz,loss,terms", [
    (64, 3, 3, O.POISSON, dict(w_pacbed=0.3, w_sparse=0.1)),
    (64, 2, 2, O.GAUSSIAN, dict(w_pacbed=0.5, p_pacbed=1.0, w_sparse=0.05, p_sparse=2.0)),
    (128, 2, 3, O.POISSON, dict(w_pacbed=0.2, w_sparse=0.1, p_sparse=0.7)),
    (256, 2, 2, O.POISSON, dict(w_pacbed=0.3, w_sparse=0.1)),
])
def test_total_loss_matches_oracle(N, M, Nz, loss, terms):
    scan = (2, 2) if N == 256 else (3, 3)
    case = make_case(N=N, M=M, Nz=Nz, scan=scan, loss=loss, seed=70 + N)
    idx = list(range(case.Ntot))[::-1]
    got_loss, g = _run(case, idx, terms)
    ref = _oracle(case, idx, terms)
    base = oracle_grads(case, idx)
    assert abs(ref.loss - base.loss) > 1e-3 * abs(base.loss)  # the extra terms matter here
    assert abs(got_loss - ref.loss) <= 1e-5 * abs(ref.loss)
    for n in NAMES:
        got = g.__dict__[n].detach().cpu().numpy()
        if n == "dz":
            # one scalar: where the PACBED part nearly cancels the likelihood part (N = 256 here:
            # their sum is 60x smaller than either), FP32 rounding is relative to the parts
            err = abs(got[0] - ref.dz) / max(abs(ref.dz), abs(base.dz))
        else:
            err = rel_l2(got, getattr(ref, n))
        assert err <= 1e-4, (n, err)


def test_split_path_total_loss():
    terms = dict(w_pacbed=0.3, w_sparse=0.1)
    case = make_case(N=64, M=2, Nz=3, scan=(3, 3), seed=81)
    idx = list(range(case.Ntot))
    got_loss, g = _run(case, idx, terms, fft="bf16x3")
    ref = _oracle(case, idx, terms)
    assert abs(got_loss - ref.loss) <= 1e-4 * abs(ref.loss)
    for n in NAMES:
        got = g.__dict__[n].detach().cpu().numpy()
        assert rel_l2(got[0] if n == "dz" else got, getattr(ref, n)) <= 1e-3, n


def test_sparse_term_without_phase_gradient():
    """The term enters the loss even when only the probe gradient is asked for."""
    terms = dict(w_sparse=0.1)
    case = make_case(N=64, M=2, Nz=2, scan=(2, 2), seed=82)
    idx = [0, 1, 2, 3]
    got_loss, g = _run(case, idx, terms, grads=("probe",))
    ref = _oracle(case, idx, terms)
    assert abs(got_loss - ref.loss) <= 1e-5 * abs(ref.loss)
    assert rel_l2(g.probe.cpu().numpy(), ref.probe) <= 1e-4
