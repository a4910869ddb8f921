"""pty_loss_grad_noalloc, the entry point that allocates nothing, agrees with pty_loss_grad.

Some callers cannot allocate device memory themselves: code running inside a host framework that
owns every device allocation through its own pool, or a real-time loop that cannot afford the
device-wide synchronisation of cudaMalloc / cudaFree.  For them the library keeps a fixed scratch
array in its own device code.  These tests call that entry point through the C ABI and compare its
loss, modelled patterns and gradients with the workspace entry point's on the same inputs, on two
calls in a row (the second call reuses the array the first one left behind).

The file name sorts last so that a run stopping at its first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

from tests.cases import make_case, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_I = 1e-5  # patterns and loss, as in the oracle parity tests
TOL_G = 1e-4  # gradients (float atomics make the last bits order dependent)
NAMES = ("amp", "phase", "probe", "pos", "tilt", "dz")


def _setup():
    from paper_2505_07814_gb300.ptycho import Geometry, Params, Ptycho

    case = make_case(N=64, M=2, Nz=3, scan=(2, 3), seed=21)
    g = case.geom
    geom = Geometry(N=g.N, M=g.M, Nz=g.Nz, H=g.H, W=g.W, Ntot=case.Ntot, dx=g.dx, lam=g.lam)
    dev = torch.device("cuda")
    f32 = dict(dtype=torch.float32, device=dev)
    params = Params(amp=torch.tensor(case.amp, **f32), phase=torch.tensor(case.phase, **f32),
                    probe=torch.tensor(case.probe, dtype=torch.complex64, device=dev),
                    pos=torch.tensor(case.pos, **f32), tilt=torch.tensor(case.tilt, **f32),
                    dz=torch.tensor([case.dz], **f32))
    I_meas = torch.tensor(case.I_meas, **f32)
    return case, geom, params, I_meas, Ptycho(geom, case.Ntot, device=dev)


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    from paper_2505_07814_gb300 import _lib

    case, geom, params, I_meas, pt = _setup()
    idx = [4, 0, 5, 2, 1, 3]
    B, N = len(idx), geom.N
    I_ref = torch.empty((B, N, N), dtype=torch.float32, device="cuda")
    loss_ref, g_ref = pt.loss_grad(params, idx, I_meas, I_model=I_ref)
    loss_ref = loss_ref.item()
    g_ref = {n: getattr(g_ref, n).clone() for n in NAMES}

    idx_t = torch.tensor(idx, dtype=torch.int32, device="cuda")
    cg = geom.c()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        grads = params.zeros_like()
        for t in (grads.amp, grads.phase, grads.pos, grads.tilt, grads.dz):
            t.fill_(5.0)  # overwritten in full (accumulate = 0)
        grads.probe.fill_(5.0)
        I_model = torch.full((B, N, N), -1.0, dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        _lib.pty_loss_grad_noalloc(cg, B, idx_t.data_ptr(), *pt._param_ptrs(params), I_meas.data_ptr(),
                                   loss.data_ptr(), I_model.data_ptr(), *pt._param_ptrs(grads), 0,
                                   status.data_ptr(), stream)
        torch.cuda.synchronize()
        assert status.item() == 0, call
        assert abs(loss.item() - loss_ref) <= TOL_I * abs(loss_ref), call
        assert rel_l2(I_model.cpu().numpy(), I_ref.cpu().numpy()) <= TOL_I, call
        for n in NAMES:
            err = rel_l2(getattr(grads, n).cpu().numpy(), g_ref[n].cpu().numpy())
            assert err <= TOL_G, (call, n, err)


def test_noalloc_rejects_batch_larger_than_its_scratch():
    from paper_2505_07814_gb300 import _lib

    g = _lib.pty_geom(N=128, M=6, Nz=8, H=512, W=512, Ntot=4096, dx=0.1, lambda_=0.0251, loss=0, p=0.0,
                      eps=1e-6, grad_mask=63, global_tilt=0)
    fake = ctypes.c_void_p(0x10000)  # never dereferenced: the size check comes first
    lib = _lib.load()
    rc = lib.pty_loss_grad_noalloc(ctypes.byref(g), 512, *([fake] * 16), 0, None, None)
    assert rc == _lib.PTY_EWORKSPACE
    assert "fixed area" in lib.pty_last_error().decode()
