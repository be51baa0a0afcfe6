"""Reference gradient: the full-linearisation adjoint of every implicit step,
solved directly (oracle; test infrastructure only).

Sec. 3, Eqns 8-12: from grad g(x) = 0,
    Hess g(x) z = (dL/dx)^T,      dL/dy = z^T M / h^2,
with Hess g = M/h^2 + Hess E (Eqn 13; Hess E from Eqn 21).  Back-propagation
through several steps repeats this for every (x, y) pair (Sec. 3).  With
y_t = x_t + h v_t + h^2 M^-1 f_t and v_{t+1} = (x_{t+1} - x_t)/h, the upstream
(dL/dx_{t+1}, dL/dv_{t+1}) gives gbar = dL/dx_{t+1} + dL/dv_{t+1}/h and
    dL/dx_t += dL/dy - dL/dv_{t+1}/h,   dL/dv_t += h dL/dy,   dL/df_t = z.
Parameter gradients follow from the implicit function theorem:
dL/dtheta = -z^T d(grad g)/dtheta, e.g. dL/dw_c = -z^T G_c^T (G_c x - p_c)
(Eqn 20 differentiated in w_c); dL/da = -w z^T G^T (d grad / da) for the
muscle actuation, and the friction force chains into (x_t, v_t, mu)
(Sec. 5.1: "compute dL/df_ext using the chain rule").
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .model import Model


def backward(model: Model, xs, vs, gx, gv=None, act=None, mu=None):
    """Back-propagate through a rollout.

    xs, vs: (T+1, n, 3) states from the forward rollout.
    gx: (T+1, n, 3) direct loss gradients dL/dx_t (zeros where the loss does
        not depend on x_t); gv likewise for velocities (None = zeros).
    Returns a dict with g_x0, g_v0 (n,3), g_fext (n,3, summed over steps),
    g_wc, g_wv, g_wm (per element, d/d weight per unit volume), g_act (T,e),
    g_mu, and per-step adjoint vectors zs (T, n, 3).
    """
    T = xs.shape[0] - 1
    n = model.mesh.n
    h = model.h
    free = model.free_nodes
    dofs = model.free_dofs
    Vq = model.mesh.Vq
    ax = np.array(gx[T], dtype=np.float64, copy=True)
    av = np.zeros((n, 3)) if gv is None else np.array(gv[T], dtype=np.float64, copy=True)
    g_fext = np.zeros((n, 3))
    g_wc = np.zeros(model.mesh.e)
    g_wv = np.zeros(model.mesh.e)
    g_wm = np.zeros(model.mesh.e)
    g_act = np.zeros((T, model.mesh.e))
    g_mu = 0.0
    zs = np.zeros((T, n, 3))
    for t in reversed(range(T)):
        a_t = None if act is None else act[t]
        gbar = (ax + av / h)[free].ravel()
        H = model.hessian(xs[t + 1], a_t)[dofs][:, dofs].tocsc()
        zf = spla.splu(H).solve(gbar)
        z = np.zeros((n, 3))
        z[free] = zf.reshape(-1, 3)
        zs[t] = z
        dLdy = model.m[:, None] * z / h ** 2
        new_ax = np.zeros((n, 3))
        new_av = np.zeros((n, 3))
        new_ax[free] = (dLdy - av / h)[free]
        new_av[free] = (h * dLdy)[free]
        g_fext += z
        fx, fv, fm = model.friction_vjp(xs[t], vs[t], z, mu)
        new_ax += fx
        new_av += fv
        g_mu += fm
        # parameter gradients at x_{t+1}
        loc = model.local(xs[t + 1], a_t)
        Gz = model.mesh.deformation_gradients(z)          # G_q z_e, (e, 8, 3, 3)
        F = loc["F"]
        if "R" in loc:
            g_wc += -Vq * np.einsum("eqij,eqij->e", Gz, F - loc["R"])
        if "D" in loc:
            g_wv += -Vq * np.einsum("eqij,eqij->e", Gz, F - loc["D"])
        if "P_nh" in loc:
            # Neo-Hookean: dP/dw_corot = (F - F^-T)/2 (mu = w_corot/2), dP/dw_vol = log J F^-T
            FinvT = np.swapaxes(np.linalg.inv(F), -1, -2)
            logJ = np.log(np.linalg.det(F))
            g_wc += -Vq * np.einsum("eqij,eqij->e", Gz, 0.5 * (F - FinvT))
            g_wv += -Vq * np.einsum("eqij,eqij->e", Gz, logJ[..., None, None] * FinvT)
        if "f" in loc:
            Gzm = np.einsum("eqij,ej->eqi", Gz, model.fiber)
            g_wm += -Vq * np.einsum("eqi,eqi->e", Gzm, loc["f"] - loc["pm"])
            fh = loc["f"] / np.linalg.norm(loc["f"], axis=2, keepdims=True)
            g_act[t] = -model.w_musc * Vq * np.einsum("eqi,eqi->e", Gzm, fh)
        ax = new_ax + gx[t]
        av = new_av + (0.0 if gv is None else gv[t])
    return {"g_x0": ax, "g_v0": av, "g_fext": g_fext, "g_wc": g_wc, "g_wv": g_wv,
            "g_wm": g_wm, "g_act": g_act, "g_mu": g_mu, "zs": zs}


def material_gradients(model: Model, grads):
    """Chain dL/dw to Young's modulus per element and Poisson's ratio through
    w_corot = E/(1+nu), w_vol = E nu/((1+nu)(1-2nu)), w_muscle = E."""
    s = model.scene
    E = model.youngs
    nu = model.poisson
    gE = np.zeros_like(E)
    gnu = 0.0
    if s.corotated:
        gE += grads["g_wc"] / (1.0 + nu)
        gnu += np.sum(grads["g_wc"] * (-E / (1.0 + nu) ** 2))
    if s.volume:
        q = (1.0 + nu) * (1.0 - 2.0 * nu)
        gE += grads["g_wv"] * nu / q
        gnu += np.sum(grads["g_wv"] * E * (1.0 + 2.0 * nu ** 2) / q ** 2)
    if s.muscle is not None:
        gE += grads["g_wm"] * np.asarray(s.muscle, dtype=np.float64)
    return gE, gnu


def final_position_loss(model: Model, xs, w):
    """L = sum(w * x_T) (Sec. 6: a random weighted sum of final positions)."""
    T = xs.shape[0] - 1
    gx = np.zeros_like(xs)
    gx[T] = w
    return float(np.sum(w * xs[T])), gx
