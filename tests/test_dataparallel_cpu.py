"""The data-parallel step's host logic (paper_2505_07814_gb300.data_parallel) on two gloo ranks.

Each rank holds one part of a batch.  The library calls are replaced, in this test only, by a
stand-in that returns the FP64 oracle's statistics and part gradients (reading R11), so that the
order of the calls, the statistics exchange and the gradient reduction are checked without a GPU:
after the step every rank must hold the whole batch's loss and gradients, and the statistics it
handed to the part call must be the whole batch's."""
import dataclasses
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(loss):
    from oracle import ptycho as O
    from tests.test_oracle import _small_problem
    return _small_problem(n_pos=5, loss=O.POISSON if loss == "poisson" else O.GAUSSIAN, seed=11)


@dataclasses.dataclass
class _Geom:
    grads: tuple = ("amp", "phase", "probe", "pos", "tilt", "dz")


class _OraclePart:
    """Stand-in for Ptycho with the two calls the data-parallel step makes, answered by the oracle
    for the part [lo, hi) of the whole batch `whole`."""

    def __init__(self, prob, whole, lo, hi):
        self.prob, self.whole, self.lo, self.hi = prob, whole, lo, hi
        self.geom = _Geom()
        self.seen_stats = None

    def loss_stats(self, params, idx, I_meas):
        from oracle import ptycho as O
        geom, amp, phase, probe, pos, tilt, dz, Im = self.prob
        assert list(idx) == self.whole[self.lo:self.hi]
        I = O.model_patterns(geom, amp, phase, probe, pos, tilt, dz, idx)
        Id = np.stack([Im[j] for j in idx])
        p = geom.power
        S = np.sum(O._pow(Id, p))
        Q = np.sum((O._pow(I, p) - O._pow(Id, p)) ** 2) if geom.loss == O.GAUSSIAN else 0.0
        return torch.tensor([S, Q, float(I.size)], dtype=torch.float64)

    def loss_grad(self, params, idx, I_meas, grads=None, whole_stats=None):
        from oracle import ptycho as O
        self.seen_stats = whole_stats.clone()
        geom, amp, phase, probe, pos, tilt, dz, Im = self.prob
        g = O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, Im, self.whole, part=(self.lo, self.hi))
        for name in ("amp", "phase", "probe", "pos", "tilt"):
            getattr(grads, name).copy_(torch.as_tensor(getattr(g, name)))
        grads.dz.fill_(g.dz)
        return torch.tensor([g.loss], dtype=torch.float64), grads


def _rank(rank, world, port, loss, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2505_07814_gb300 import data_parallel as DP
    from paper_2505_07814_gb300.ptycho import Params
    prob = _problem(loss)
    geom, amp, phase, probe, pos, tilt, dz, I_meas = prob
    whole = [3, 0, 4, 1, 2]
    mine = DP.split(whole, rank, world)
    lo = whole.index(mine[0])
    pt = _OraclePart(prob, whole, lo, lo + len(mine))
    zeros = Params(amp=torch.zeros(amp.shape, dtype=torch.float64), phase=torch.zeros(phase.shape, dtype=torch.float64),
                   probe=torch.zeros(probe.shape, dtype=torch.complex128),
                   pos=torch.zeros(pos.shape, dtype=torch.float64), tilt=torch.zeros(np.shape(tilt), dtype=torch.float64),
                   dz=torch.zeros(1, dtype=torch.float64))
    loss_t, grads = DP.loss_grad(pt, None, mine, None, zeros, dist.all_reduce)
    q.put((rank, float(loss_t[0]), {n: getattr(grads, n).numpy().copy() for n in DP.GRAD_NAMES},
           pt.seen_stats.numpy()))
    dist.destroy_process_group()


@pytest.mark.parametrize("loss", ["poisson", "gaussian"])
def test_two_ranks_reproduce_the_whole_batch(loss):
    from oracle import ptycho as O
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, loss, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    geom, amp, phase, probe, pos, tilt, dz, I_meas = _problem(loss)
    whole = [3, 0, 4, 1, 2]
    ref = O.loss_and_grad(geom, amp, phase, probe, pos, tilt, dz, I_meas, whole)
    I = O.model_patterns(geom, amp, phase, probe, pos, tilt, dz, whole)
    Id = np.stack([I_meas[j] for j in whole])
    p_ = geom.power
    S = np.sum(O._pow(Id, p_))
    Q = np.sum((O._pow(I, p_) - O._pow(Id, p_)) ** 2) if geom.loss == O.GAUSSIAN else 0.0
    for rank, L, g, seen in out:
        np.testing.assert_allclose(seen, [S, Q, I.size], rtol=1e-12)  # the whole batch's statistics
        assert np.isclose(L, ref.loss, rtol=1e-12)
        for name in ("amp", "phase", "probe", "pos", "tilt"):
            r = getattr(ref, name)
            assert np.linalg.norm((g[name] - r).ravel()) <= 1e-12 * np.linalg.norm(r.ravel()), (rank, name)
        assert np.isclose(g["dz"][0], ref.dz, rtol=1e-11)
