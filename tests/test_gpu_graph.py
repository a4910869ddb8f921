"""pty_loss_grad captured into a CUDA graph: the replay matches the eager call and reads the live
parameter buffers (no host synchronisation or allocation inside a call)."""
import numpy as np
import pytest

from tests.cases import make_case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ("amp", "phase", "probe", "pos", "tilt", "dz")


def _setup():
    from paper_2505_07814_gb300.ptycho import Geometry, Params, Ptycho
    case = make_case(N=64, M=2, Nz=3, scan=(3, 4), seed=21)
    g = case.geom
    geom = Geometry(N=g.N, M=g.M, Nz=g.Nz, H=g.H, W=g.W, Ntot=case.Ntot, dx=g.dx, lam=g.lam)
    dev = torch.device("cuda")
    f32 = dict(dtype=torch.float32, device=dev)
    params = Params(amp=torch.tensor(case.amp, **f32), phase=torch.tensor(case.phase, **f32),
                    probe=torch.tensor(case.probe, dtype=torch.complex64, device=dev),
                    pos=torch.tensor(case.pos, **f32), tilt=torch.tensor(case.tilt, **f32),
                    dz=torch.tensor([case.dz], **f32))
    return Ptycho(geom, case.Ntot, device=dev), params, torch.tensor(case.I_meas, **f32), case


def _snapshot(loss, grads):
    return [loss.item()] + [getattr(grads, n).detach().cpu().numpy().copy() for n in NAMES]


def _close(a, b, tol=1e-5):
    assert abs(a[0] - b[0]) <= tol * abs(b[0])
    for x, y, n in zip(a[1:], b[1:], NAMES):
        assert rel_l2(x, y) <= tol, n


def test_loss_grad_replays_from_a_cuda_graph():
    pt, params, I_meas, case = _setup()
    idx = torch.tensor([5, 0, 11, 3, 7, 1], dtype=torch.int32, device="cuda")
    grads = params.zeros_like()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up on a side stream, as graph capture requires
        pt.loss_grad(params, idx, I_meas, grads=grads)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    eager = _snapshot(*pt.loss_grad(params, idx, I_meas, grads=params.zeros_like()))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        loss, out = pt.loss_grad(params, idx, I_meas, grads=grads)
    graph.replay()
    torch.cuda.synchronize()
    assert pt.status() == 0
    _close(_snapshot(loss, out), eager)
    # the graph reads the parameter buffers as they are at replay time
    params.amp.mul_(1.01)
    params.pos.add_(0.1)
    graph.replay()
    torch.cuda.synchronize()
    replayed = _snapshot(loss, out)
    eager2 = _snapshot(*pt.loss_grad(params, idx, I_meas, grads=params.zeros_like()))
    _close(replayed, eager2)
    assert abs(replayed[0] - eager[0]) > 1e-6 * abs(eager[0])
