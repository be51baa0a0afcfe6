"""PyTorch autograd over the differentiable PD rollout.

`Simulator.rollout(x0, v0, T, ...)` returns the trajectories (x_t, v_t),
t = 0..T (with opts checkpoint_every = K > 0: the checkpointed states t = 0, K,
2K, ..., T; the others are recomputed in the backward pass), as tensors that carry gradients to x0, v0, f_ext, the actuation, the
material weights (w_corot, w_vol, w_muscle) and the friction coefficient mu.  The
forward pass is pd_forward (Alg. 1 with L-BFGS); the backward pass is one
pd_backward call with the loss gradients of every state (Sec. 4: the adjoint
splitting iteration, Alg. 2, per step, chained through Eqns 10-12).  The mesh is
refactorised only when the weight tensors change.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import _native as N
from . import api


class Simulator:
    """A voxel mesh resident on one GPU plus its current factorisation."""

    def __init__(self, mesh: api.PDMesh, h: float, gravity=(0.0, 0.0, -9.81), k_contact: float = 0.0,
                 precision: int = N.PD_PREC_FP64, opts: Optional[dict] = None):
        self.mesh = mesh
        self.h = h
        self.gravity = tuple(gravity)
        self.k_contact = k_contact
        self.precision = precision
        self.opts = dict(opts or {})
        self._key = None
        self._held = None

    @classmethod
    def from_scene(cls, sc, precision=N.PD_PREC_FP64, opts=None, device=0):
        mesh = api.PDMesh.from_scene(sc, device=device)
        return cls(mesh, sc.h, tuple(sc.gravity), sc.k_contact, precision, opts)

    @staticmethod
    def _tag(t):
        return None if t is None else (t.data_ptr(), t._version, tuple(t.shape))

    def ensure_factor(self, w_corot, w_vol, w_muscle, fiber):
        # The key is (address, version, shape) of the tensors the factor was built
        # from; holding those tensors keeps their memory from being handed to new
        # tensors, so a new weight tensor always has a new key.
        key = tuple(self._tag(t) for t in (w_corot, w_vol, w_muscle, fiber))
        if key != self._key:
            self.mesh.factorize(w_corot, w_vol, w_muscle, fiber, h=self.h, gravity=self.gravity,
                                k_contact=self.k_contact, precision=self.precision)
            self._key = key
            self._held = (w_corot, w_vol, w_muscle, fiber)

    def rollout(self, x0, v0, T: int, f_ext=None, act=None, w_corot=None, w_vol=None, w_muscle=None,
                fiber=None, mu=None):
        """(x, v): (S, n, 3) each, S = T+1, or T/K+1 checkpointed states with opts
        checkpoint_every = K > 0.  mu: Python float or 0-dim tensor."""
        if mu is None:
            mu = 0.0
        mu_t = mu if torch.is_tensor(mu) else torch.tensor(float(mu), dtype=torch.float64, device=x0.device)
        return _Rollout.apply(self, T, fiber, x0, v0, f_ext, act, w_corot, w_vol, w_muscle, mu_t)


def _c(t):
    return None if t is None else t.detach().contiguous()


def _every_state(g, T, K):
    """(T+1, n, 3) loss gradient from the gradient of the returned states, which
    are every state (K <= 0) or the checkpoints 0, K, 2K, ... (K > 0)."""
    if K <= 0:
        return g.contiguous()
    full = g.new_zeros((T + 1,) + tuple(g.shape[1:]))
    full[::K] = g
    return full


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sim, T, fiber, x0, v0, f_ext, act, w_corot, w_vol, w_muscle, mu):
        x0, v0, f_ext, act = _c(x0), _c(v0), _c(f_ext), _c(act)
        wc, wv, wm = _c(w_corot), _c(w_vol), _c(w_muscle)
        fib = _c(fiber)
        sim.ensure_factor(wc, wv, wm, fib)
        opts = api.solver_opts(**sim.opts)
        roll = sim.mesh.forward(x0, v0, T, f_ext=f_ext, act=act, mu=float(mu), opts=opts)
        ctx.sim, ctx.T, ctx.K = sim, T, roll.checkpoint_every
        ctx.has = tuple(t is not None for t in (f_ext, act, w_corot, w_vol, w_muscle))
        ctx.save_for_backward(roll.x, roll.v, f_ext if f_ext is not None else roll.x.new_empty(0),
                              act if act is not None else roll.x.new_empty(0), wc, wv, wm, fib, mu)
        return roll.x, roll.v

    @staticmethod
    def backward(ctx, gx, gv):
        sim, T = ctx.sim, ctx.T
        xs, vs, f_ext, act, wc, wv, wm, fib, mu = ctx.saved_tensors
        has_f, has_a = ctx.has[0], ctx.has[1]
        f_ext = f_ext if has_f else None
        act = act if has_a else None
        # the factor may have been replaced by another rollout since the forward pass
        sim.ensure_factor(wc, wv, wm, fib)
        if gx is None:
            gx = torch.zeros_like(xs)
        # with checkpointing the forward output holds states 0, K, 2K, ... only: their
        # gradients go to those steps of the (T+1)-state loss gradient, zeros elsewhere
        K = ctx.K
        gx = _every_state(gx, T, K)
        gv = None if gv is None else _every_state(gv, T, K)
        need = ctx.needs_input_grad
        names = [(3, "x0"), (4, "v0"), (5, "fext"), (6, "act"), (7, "w_corot"), (8, "w_vol"), (9, "w_muscle"),
                 (10, "mu")]
        want = tuple(name for i, name in names if need[i])
        roll = api.Rollout(xs, vs, {}, N.PD_OK, K)
        opts = api.solver_opts(**sim.opts)
        out = sim.mesh.backward(roll, T, gx, dL_dv=gv, loss_all_steps=True, f_ext=f_ext, act=act, mu=float(mu),
                                opts=opts, want=want)
        g = {name: out.get(name) for _, name in names}
        gmu = g["mu"].reshape(()) if g["mu"] is not None else None
        return (None, None, None, g["x0"], g["v0"], g["fext"], g["act"], g["w_corot"], g["w_vol"], g["w_muscle"],
                gmu)
