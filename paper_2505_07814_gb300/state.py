"""Checkpoint and resume of a reconstruction: the six optimisable parameters (object amplitude and
phase, probe modes, positions, tilts, dz; Sec. "AD-optimizable parameters"), the Adam state that
updates them (first and second moments, step count, learning rates, betas, eps) and the iteration
counter, written to one file and read back onto a device.  A resumed run continues the same
trajectory: the next Adam step sees the same parameters, moments and bias-correction count.

The file is a torch.save dictionary of CPU tensors plus plain Python values, so it can be read on
any machine; nothing in it depends on the library build.
"""
from __future__ import annotations

import dataclasses

import torch

from .ptycho import GRAD_BITS, Adam, Geometry, Params

FORMAT = "pty-reconstruction-state-1"
NAMES = ("amp", "phase", "probe", "pos", "tilt", "dz")


def save(path: str, geom: Geometry, params: Params, adam: Adam | None = None, iteration: int = 0,
         extra: dict | None = None) -> None:
    """Write the reconstruction state to `path` (parameters copied to host memory)."""
    state = {"format": FORMAT, "geometry": dataclasses.asdict(geom), "iteration": int(iteration),
             "params": {n: getattr(params, n).detach().cpu().clone() for n in NAMES}, "extra": dict(extra or {})}
    if adam is not None:
        state["adam"] = {"m": {n: getattr(adam.m, n).detach().cpu().clone() for n in NAMES},
                         "v": {n: getattr(adam.v, n).detach().cpu().clone() for n in NAMES},
                         "t": int(adam.t), "lr": dict(adam.lr), "betas": tuple(adam.betas), "eps": float(adam.eps)}
    torch.save(state, path)


def load(path: str, device="cuda"):
    """Read a state written by `save`.  Returns (geometry, params, adam or None, iteration, extra),
    with the tensors on `device`."""
    state = torch.load(path, map_location="cpu", weights_only=False)
    if state.get("format") != FORMAT:
        raise ValueError("%s is not a reconstruction state (format %r)" % (path, state.get("format")))
    g = dict(state["geometry"])
    g["grads"] = tuple(g["grads"])
    geom = Geometry(**g)
    params = Params(*(state["params"][n].to(device) for n in NAMES))
    adam = None
    if "adam" in state:
        a = state["adam"]
        adam = Adam(params, {k: a["lr"][k] for k in GRAD_BITS}, betas=tuple(a["betas"]), eps=a["eps"])
        for n in NAMES:
            getattr(adam.m, n).copy_(a["m"][n].to(device))
            getattr(adam.v, n).copy_(a["v"][n].to(device))
        adam.t = a["t"]
    return geom, params, adam, state["iteration"], state["extra"]
