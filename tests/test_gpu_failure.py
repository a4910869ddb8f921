"""Failure detection without a GPU fault: device status bits read back through the C ABI.

- A non-finite measured pattern reaches the loss: the call still runs to its end and
  PTY_ENONFINITE is set in the status word (pty_status).
- A bounded device wait runs out: the tensor-core GEMM's pipeline waits are given a poll limit of
  0 (pty_set_wait_limit), so each gives up at once; the kernel sets PTY_ETIMEOUT, waits for the
  matrix products it already issued, releases its tensor memory and returns.  The limit is then
  restored and the next call on the same context runs clean and matches the oracle.
No test here faults, traps or hangs the GPU: the waits that run out are the ones whose give-up path
drains before it releases anything.
"""
import numpy as np
import pytest

from tests.cases import make_case, oracle_grads, rel_l2
from tests.test_gpu_parity import _gpu, _np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_nonfinite_measured_pattern_sets_enonfinite():
    from paper_2505_07814_gb300 import _lib
    case = make_case(N=64, M=2, Nz=2, scan=(2, 2), seed=31)
    pt, params, I_meas = _gpu(case)
    bad = I_meas.clone()
    bad[2, 10, 17] = float("nan")
    loss, _ = pt.loss_grad(params, [0, 2, 3], bad)
    st = pt.status()
    assert st & _lib.PTY_ENONFINITE, st
    assert not st & _lib.PTY_ETIMEOUT
    # a batch that does not read the bad pattern is clean again (the word is cleared per call)
    loss, _ = pt.loss_grad(params, [0, 1, 3], bad)
    assert pt.status() == 0 and np.isfinite(loss.item())


def test_gemm_wait_that_runs_out_returns_etimeout_and_the_next_call_is_clean():
    from paper_2505_07814_gb300 import _lib
    from tests.test_gpu_split import _gpu as _gpu_split
    case = make_case(N=64, M=2, Nz=2, scan=(2, 2), seed=33)
    idx = [0, 1, 2, 3]
    pt, params, I_meas = _gpu_split(case, "fp16")
    pt.loss_grad(params, idx, I_meas)  # first call builds the DFT tables
    assert pt.status() == 0
    try:
        _lib.pty_set_wait_limit(0)
        pt.loss_grad(params, idx, I_meas)
        st = pt.status()
    finally:
        _lib.pty_set_wait_limit(-1)
    assert st >= 0 and st & _lib.PTY_ETIMEOUT, st
    # same context, default limit: a clean call that matches the oracle
    I_model = torch.empty((len(idx), 64, 64), dtype=torch.float32, device="cuda")
    loss, g = pt.loss_grad(params, idx, I_meas, I_model=I_model)
    assert pt.status() == 0
    ref = oracle_grads(case, idx)
    assert rel_l2(_np(I_model), ref.I_model) <= 1e-4
    assert rel_l2(_np(g.amp), ref.amp) <= 1e-3
    # the FP32 path on the same context is unaffected
    pt32, params32, I32 = _gpu(case)
    pt32.loss_grad(params32, idx, I32)
    assert pt32.status() == 0
