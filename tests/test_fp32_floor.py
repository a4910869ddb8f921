"""The single-precision evaluation used to measure FP32 error floors (tests/fp32_floor.py) computes
the same gradients as the FP64 oracle, to single-precision accuracy, on a small problem."""
import numpy as np

from oracle import ptycho as O
from tests.fp32_floor import object_gradients_fp32
from tests.test_oracle import _small_problem


def test_fp32_evaluation_agrees_with_the_oracle_to_single_precision():
    geom, amp, phase, probe, pos, tilt, dz, I_meas = _small_problem(n_pos=4, seed=8)
    idx = [2, 0, 3, 1]
    ref = O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx)
    ga, gp = object_gradients_fp32(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx)
    for got, exp in ((ga, ref.amp), (gp, ref.phase)):
        err = np.linalg.norm(got - exp) / np.linalg.norm(exp)
        assert 1e-9 < err < 1e-5, err  # single-precision rounding, not a formula difference
