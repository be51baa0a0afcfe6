"""Second CPU forward/backward for meshes where the Newton oracle is too slow
(oracle; test infrastructure only).

Forward: Projective Dynamics (Alg. 1) accelerated by L-BFGS with the constant
matrix A as initial Hessian (Sec. 4, "Further acceleration with quasi-Newton
methods", after Liu et al. 2017) and an Armijo line search (at most 10 tries,
Sec. 6).  Plain PD is the special case of an empty history and unit steps:
x <- x - A^-1 grad g(x) equals x <- A^-1 (M y/h^2 + sum w G^T p) (Eqn 19).
It converges to the same implicit-Euler fixed point grad g = 0 as Newton
(Sec. 3, the PD solution is a critical point of g).

Backward: the adjoint system Hess g z = dL/dx (Eqn 12) solved by MINRES with
the SPD preconditioner A^-1 (Hess g = A - Delta A, Eqn 22), to a tight
relative residual.

A = I_3 (x) L_A: the scalar matrix L_A over the free nodes is factored once
with SuperLU and applied to the three coordinate columns.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .model import Model


class ScalarA:
    """Factor of the free-node block of L_A (the x-coordinate block of A)."""

    def __init__(self, model: Model):
        A = model.A_matrix()
        xdofs = model.free_nodes * 3
        self.LA = A[xdofs][:, xdofs].tocsc()
        self.lu = spla.splu(self.LA)

    def solve(self, r):
        """A^-1 r for r of shape (n_free*3,) (node-major)."""
        R = np.asarray(r).reshape(-1, 3)
        return self.lu.solve(np.ascontiguousarray(R)).reshape(-1)


def pd_lbfgs_step(model: Model, Afac: ScalarA, x, v, f_ext, act=None, mu=None, tol=1e-12,
                  history=5, max_iter=2000, stop=None):
    """One implicit-Euler step by PD + L-BFGS from the predictor; `stop(iters)`,
    when given, is called after every iteration and ends the step early when it
    returns True (used to time a bounded number of iterations)."""
    free = model.free_nodes
    y = model.predictor(x, v, f_ext, mu)
    xn = np.array(y, copy=True)
    xn[model.dirichlet] = model.mesh.X[model.dirichlet]
    loc = model.local(xn, act)
    gval = model.g_value(xn, y, act, loc)
    gr = model.grad_g(xn, y, act, loc)
    ref = max(np.linalg.norm(gr), np.linalg.norm((model.m[:, None] * y / model.h ** 2)[free]))
    S, Y = [], []
    it = 0
    while np.linalg.norm(gr) > tol * ref and it < max_iter:
        q = gr.copy()
        alphas = []
        for s, yv in zip(reversed(S), reversed(Y)):
            a = (s @ q) / (yv @ s)
            q -= a * yv
            alphas.append(a)
        r = Afac.solve(q)
        for (s, yv), a in zip(zip(S, Y), reversed(alphas)):
            b = (yv @ r) / (yv @ s)
            r += s * (a - b)
        d = -r
        slope = d @ gr
        if slope >= 0:                       # not a descent direction: plain PD step
            S, Y = [], []
            d = -Afac.solve(gr)
            slope = d @ gr
        alpha = 1.0
        for _ in range(10):
            xt = np.array(xn, copy=True)
            xt[free] += alpha * d.reshape(-1, 3)
            loct = model.local(xt, act)
            gt = model.g_value(xt, y, act, loct)
            if gt <= gval + 1e-4 * alpha * slope + 1e-14 * abs(gval):
                break
            alpha *= 0.5
        grt = model.grad_g(xt, y, act, loct)
        s = (xt - xn)[free].ravel()
        yv = grt - gr
        if s @ yv > 0:
            S.append(s)
            Y.append(yv)
            if len(S) > history:
                S.pop(0)
                Y.pop(0)
        xn, gr, gval = xt, grt, gt
        it += 1
        if stop is not None and stop(it):
            break
    vn = (xn - x) / model.h
    return xn, vn, {"iters": it, "residual": float(np.linalg.norm(gr)), "ref": float(ref)}


def rollout(model: Model, x0, v0, f_ext, act=None, T=None, mu=None, tol=1e-12):
    T = model.scene.T if T is None else T
    Afac = ScalarA(model)
    xs = [np.array(x0, dtype=np.float64)]
    vs = [np.array(v0, dtype=np.float64)]
    infos = []
    for t in range(T):
        a_t = None if act is None else act[t]
        xn, vn, info = pd_lbfgs_step(model, Afac, xs[-1], vs[-1], f_ext, a_t, mu, tol)
        xs.append(xn)
        vs.append(vn)
        infos.append(info)
    return np.stack(xs), np.stack(vs), infos


def adjoint_solve_minres(model: Model, Afac: ScalarA, x_next, gbar, act=None, rtol=1e-12):
    """z with Hess g(x_next) z = gbar on the free DoFs, by A^-1-preconditioned MINRES."""
    dofs = model.free_dofs
    H = model.hessian(x_next, act)[dofs][:, dofs].tocsr()
    P = spla.LinearOperator(H.shape, matvec=Afac.solve, dtype=np.float64)
    z, info = spla.minres(H, gbar, M=P, rtol=rtol, maxiter=5000)
    if info != 0:
        raise RuntimeError(f"MINRES did not converge (info={info})")
    return z
