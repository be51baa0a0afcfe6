"""Reference forward: implicit Euler solved by Newton's method with a sparse
direct solve (oracle; test infrastructure only).

Sec. 3, Eqns 1-7: x_{i+1} = x_i + h v_{i+1}; the step solves
grad g(x) = M (x - y)/h^2 - f_int(x) = 0 with y = x_i + h v_i + h^2 M^-1 f_ext.
Newton: Hess g(x^k) dx = -grad g(x^k), with a definiteness fix (fall back to
the direction -A^-1 grad g when the Newton direction is not a descent
direction) and an Armijo backtracking line search (c1 = 1e-4, halving, at
most 10 tries; Sec. 6 caps line searches at 10).  Iterations start from
x = y (Alg. 1) and stop once |grad g|_2 <= tol * max(|grad g(x^0)|_2,
|M y / h^2|_2) (reading: the paper leaves the norm unstated).  Dirichlet
nodes stay at their rest positions.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .model import Model


def _free_block(Mat, dofs):
    return Mat[dofs][:, dofs].tocsc()


def newton_step(model: Model, x, v, f_ext, act=None, mu=None, tol=1e-12, max_iter=60):
    """One implicit-Euler step.  Returns (x_next, v_next, info)."""
    free = model.free_nodes
    dofs = model.free_dofs
    y = model.predictor(x, v, f_ext, mu)
    xn = np.array(y, copy=True)
    xn[model.dirichlet] = model.mesh.X[model.dirichlet]
    gr = model.grad_g(xn, y, act)
    ref = max(np.linalg.norm(gr),
              np.linalg.norm((model.m[:, None] * y / model.h ** 2)[free]))
    A_lu = None
    it = 0
    ls_total = 0
    while np.linalg.norm(gr) > tol * ref and it < max_iter:
        H = _free_block(model.hessian(xn, act), dofs)
        try:
            dx = spla.splu(H).solve(-gr)
            ok = np.all(np.isfinite(dx)) and dx @ gr < 0
        except RuntimeError:
            ok = False
        if not ok:
            if A_lu is None:
                A_lu = spla.splu(_free_block(model.A_matrix(), dofs))
            dx = A_lu.solve(-gr)
        g0 = model.g_value(xn, y, act)
        slope = dx @ gr
        alpha = 1.0
        for _ in range(10):
            xt = np.array(xn, copy=True)
            xt[free] += alpha * dx.reshape(-1, 3)
            gt = model.g_value(xt, y, act)
            if gt <= g0 + 1e-4 * alpha * slope + 1e-14 * abs(g0):
                break
            alpha *= 0.5
            ls_total += 1
        xn = xt
        gr = model.grad_g(xn, y, act)
        it += 1
    vn = (xn - x) / model.h
    info = {"iters": it, "residual": float(np.linalg.norm(gr)), "ref": float(ref),
            "line_search": ls_total, "y": y}
    return xn, vn, info


def rollout(model: Model, x0, v0, f_ext, act=None, T=None, mu=None, tol=1e-12):
    """Forward rollout of T steps.  Returns (xs (T+1,n,3), vs (T+1,n,3), infos)."""
    T = model.scene.T if T is None else T
    xs = [np.array(x0, dtype=np.float64)]
    vs = [np.array(v0, dtype=np.float64)]
    infos = []
    for t in range(T):
        a_t = None if act is None else act[t]
        xn, vn, info = newton_step(model, xs[-1], vs[-1], f_ext, a_t, mu, tol)
        xs.append(xn)
        vs.append(vn)
        infos.append(info)
    return np.stack(xs), np.stack(vs), infos
