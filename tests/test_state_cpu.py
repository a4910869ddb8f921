"""Checkpoint and resume of a reconstruction (paper_2505_07814_gb300/state.py): the saved file
round-trips every parameter, the Adam moments and counters, the geometry and the iteration
exactly, on the CPU."""
import pytest

torch = pytest.importorskip("torch")


def test_state_round_trip(tmp_path):
    from paper_2505_07814_gb300 import state
    from paper_2505_07814_gb300.ptycho import Adam, Geometry, Params
    g = torch.Generator().manual_seed(3)
    geom = Geometry(N=64, M=2, Nz=3, H=90, W=100, Ntot=12, dx=0.1, lam=0.0251, loss="gaussian", ckpt_stride=2,
                    grads=("amp", "phase", "probe"), w_sparse=0.1)
    params = Params(amp=torch.rand(3, 90, 100, generator=g), phase=torch.rand(3, 90, 100, generator=g),
                    probe=torch.randn(2, 64, 64, dtype=torch.complex64, generator=g),
                    pos=torch.rand(12, 2, generator=g), tilt=torch.rand(12, 2, generator=g), dz=torch.tensor([2.0]))
    adam = Adam(params, {"amp": 1e-3, "phase": 3e-3, "probe": 1e-2}, betas=(0.8, 0.99), eps=1e-7)
    for n in ("amp", "phase", "probe", "pos", "tilt", "dz"):
        getattr(adam.m, n).copy_(torch.randn(getattr(params, n).shape, generator=g).to(getattr(params, n).dtype))
        getattr(adam.v, n).copy_(torch.rand(getattr(params, n).shape, generator=g).to(getattr(params, n).dtype))
    adam.t = 17
    path = str(tmp_path / "rec.pt")
    state.save(path, geom, params, adam, iteration=5, extra={"loss_history": [1.0, 0.5]})
    geom2, params2, adam2, it, extra = state.load(path, device="cpu")
    assert geom2 == geom and it == 5 and extra == {"loss_history": [1.0, 0.5]}
    for n in ("amp", "phase", "probe", "pos", "tilt", "dz"):
        assert torch.equal(getattr(params2, n), getattr(params, n)), n
        assert torch.equal(getattr(adam2.m, n), getattr(adam.m, n)), n
        assert torch.equal(getattr(adam2.v, n), getattr(adam.v, n)), n
    assert adam2.t == 17 and adam2.lr == adam.lr and adam2.betas == adam.betas and adam2.eps == adam.eps
    # a file of something else is refused
    torch.save({"format": "other"}, str(tmp_path / "x.pt"))
    with pytest.raises(ValueError):
        state.load(str(tmp_path / "x.pt"), device="cpu")
