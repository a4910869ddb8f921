"""The chunked, multi-process evaluation of the oracle (tests/oracle_pool.py) equals the plain
single call on the whole batch: the Poisson normaliser rescaling is exact."""
import numpy as np

from oracle import ptycho as O
from tests.oracle_pool import poisson_loss_and_grad
from tests.test_oracle import _small_problem


def test_chunked_oracle_equals_the_whole_batch():
    geom, amp, phase, probe, pos, tilt, dz, I_meas = _small_problem(n_pos=5, seed=4)
    idx = [3, 0, 4, 2, 1]
    ref = O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx)
    got = poisson_loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, idx, procs=3)
    assert np.isclose(got.loss, ref.loss, rtol=1e-12)
    np.testing.assert_allclose(got.I_model, ref.I_model, rtol=1e-13)
    for n in ("amp", "phase", "probe", "pos", "tilt"):
        r = getattr(ref, n)
        assert np.linalg.norm((getattr(got, n) - r).ravel()) <= 1e-12 * np.linalg.norm(r.ravel()), n
    assert np.isclose(got.dz, ref.dz, rtol=1e-11)
