"""System identification by gradient-based optimisation through the simulator.

The paper's parameter-estimation experiments (Sec. 7) recover material
parameters from an observed motion by minimising a trajectory loss with L-BFGS,
with the gradients from the differentiable simulation.  Here the parameters are
log E (one value or one per element) and log nu; the loss is the mean squared
distance between the simulated and the observed positions over all states; every
evaluation refactorises A for the new weights (pd_factorize) and runs one forward
rollout and one backward pass (pd_forward / pd_backward through autograd.py).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import torch

from . import _native as N
from .autograd import Simulator


@dataclass
class SysIdResult:
    log_E: np.ndarray
    log_nu: float
    loss_history: list = field(default_factory=list)
    evaluations: int = 0


def _weights(log_E: torch.Tensor, log_nu: torch.Tensor):
    E = torch.exp(log_E)
    nu = torch.exp(log_nu)
    return E / (1.0 + nu), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def trajectory_loss(sim: Simulator, log_E, log_nu, x0, v0, T, x_obs, f_ext=None, corotated=True, volume=True):
    """mean over states and DoFs of (x_t - x_obs_t)^2 for t = 1..T."""
    wc, wv = _weights(log_E, log_nu)
    x, _ = sim.rollout(x0, v0, T, f_ext=f_ext, w_corot=wc if corotated else None, w_vol=wv if volume else None)
    return ((x[1:] - x_obs[1:]) ** 2).mean()


def identify(sc, x_obs: torch.Tensor, log_E0, log_nu0: float, T: Optional[int] = None,
             iters: int = 20, precision: int = N.PD_PREC_MIXED, opts: Optional[dict] = None,
             per_element: bool = False, device: int = 0) -> SysIdResult:
    """L-BFGS (torch.optim.LBFGS with strong-Wolfe line search) on (log E, log nu)
    of scene `sc` (a workloads.Scene: geometry, density, initial state, loads) to
    match the observed positions x_obs ((T+1, n, 3), device).  log E is one value
    for the whole body, or one per element with per_element=True."""
    T = sc.T if T is None else T
    dev = torch.device(f"cuda:{device}")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    sim = Simulator.from_scene(sc, precision=precision, opts=opts or dict(tol_fwd=1e-9, tol_bwd=1e-9,
                                                                            max_iter_fwd=3000,
                                                                            max_iter_bwd=3000),
                               device=device)
    shape = (sc.n_elems,) if per_element else ()
    log_E = t(np.broadcast_to(np.asarray(log_E0, dtype=np.float64), shape)).clone().requires_grad_(True)
    log_nu = torch.tensor(float(log_nu0), dtype=torch.float64, device=dev, requires_grad=True)
    ones = torch.ones(sc.n_elems, dtype=torch.float64, device=dev)
    x0, v0, f_ext = t(sc.x0), t(sc.v0), t(sc.f_ext)
    res = SysIdResult(log_E=np.empty(0), log_nu=0.0)
    opt = torch.optim.LBFGS([log_E, log_nu], lr=1.0, max_iter=iters, history_size=10,
                            line_search_fn="strong_wolfe", tolerance_grad=1e-14, tolerance_change=1e-16)

    scale = []   # the loss is divided by its value at the start (a constant factor):
                 # absolute trajectory errors are ~1e-10 m^2, too small for the
                 # optimiser's default step and tolerances

    def closure():
        opt.zero_grad()
        loss = trajectory_loss(sim, log_E * ones, log_nu, x0, v0, T, x_obs, f_ext, sc.corotated, sc.volume)
        if not scale:
            scale.append(max(float(loss.detach()), 1e-300))
        res.evaluations += 1
        res.loss_history.append(float(loss.detach()))
        scaled = loss / scale[0]
        scaled.backward()
        return scaled

    opt.step(closure)
    res.log_E = np.atleast_1d(log_E.detach().cpu().numpy())
    res.log_nu = float(log_nu.detach())
    sim.mesh.close()
    return res
