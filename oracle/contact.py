"""Complementarity contact (Sec. 5.2): the global step with a fixed contact set.

Oracle -- test infrastructure only (tests, smoke and the benchmark's CPU leg
may use it; the CUDA path never does).

With the contact set C fixed, every node j in C is held at its target x*_j and the
other free nodes solve the reduced system of the global step (Alg. 3):
    x_C = x*,   A_{C'C'} x_{C'} = b_{C'}          (C' = free nodes not in C)
with A = I_3 (x) L_A acting identically on the three coordinates.  The paper
evaluates this with a low-rank update of the prefactorised A (Alg. 4); the
oracle writes out the plain definition: a sparse direct solve of the reduced
matrix.  `woodbury_solve` restates Alg. 4's steps (dense, small meshes only) so
that a test can check the two against each other.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def constrained_solve(L, C, xstar, b):
    """L: scalar free-node matrix (nf x nf, sparse); C: free-node indices (c,);
    xstar: (c, 3); b: (nf, 3).  Returns x (nf, 3)."""
    nf = L.shape[0]
    C = np.asarray(C, dtype=np.int64)
    keep = np.setdiff1d(np.arange(nf), C)
    x = np.zeros((nf, 3))
    x[C] = xstar
    if keep.size:
        Lkk = L.tocsr()[keep][:, keep].tocsc()
        x[keep] = spla.splu(Lkk).solve(np.ascontiguousarray(b[keep]))
    return x


def woodbury_solve(Ld, C, xstar, b):
    """Alg. 4 as stated (dense): B1 = A^-1 I_{I x C}, B2 = I_{I x C} - B1 A_CC,
    B3 = (B1, B2), B4 = I - V P^T B3, a1 = A^-1 b, a2 = (b^T B2, b^T B1),
    a3 = B4^-1 a2^T, x = a1 + B3 a3, then x_C = x*.  Ld: dense nf x nf."""
    nf = Ld.shape[0]
    C = np.asarray(C, dtype=np.int64)
    c = C.size
    Ainv = np.linalg.inv(Ld)
    I_C = np.zeros((nf, c))
    I_C[C, np.arange(c)] = 1.0
    B1 = Ainv @ I_C
    B2 = I_C - B1 @ Ld[np.ix_(C, C)]
    B3 = np.hstack([B1, B2])
    # V P^T: rows (0 | A_{C, C'}) then (I | 0), in the original node order
    notC = np.ones(nf, dtype=bool)
    notC[C] = False
    VPt = np.zeros((2 * c, nf))
    VPt[:c][:, notC] = Ld[np.ix_(C, np.flatnonzero(notC))]
    VPt[c:, C] = np.eye(c)
    B4 = np.eye(2 * c) - VPt @ B3
    a1 = Ainv @ b
    a2 = np.vstack([B2.T @ b, B1.T @ b])
    a3 = np.linalg.solve(B4, a2)
    x = a1 + B3 @ a3
    x[C] = xstar
    return x


# ------------------------------------------------------------------ time step
# Alg. 3 on the ground z = 0 (phi(x) = z), with static friction (sticky contact).
# Readings (the paper leaves them open): a candidate whose ray x_t + s v_t,
# 0 < s <= h, reaches z = 0 is held at that intersection ("ray"; its height is 0
# by the choice of s and is stored as exactly 0, so that the next step sees the
# node touching instead of a rounding residue of either sign); a candidate
# already touching (z_t <= 0) or added later because it penetrates is held at
# (x_t, y_t, 0) ("drop").  Both targets depend on the start of the step only.
# The contact set is updated until stable: nodes whose contact force
# r_j = [M (x - y)/h^2 + grad E]_j has r_jz < 0 leave, penetrating candidates
# (z_j < 0) join.  Penalty contact and friction are off in this model.

def contact_target(xt, vt, h, rule):
    """x* of one node; rule 'ray' or 'drop'."""
    if rule == "ray":
        s = xt[2] / (-vt[2])
        return np.array([xt[0] + s * vt[0], xt[1] + s * vt[1], 0.0])
    return np.array([xt[0], xt[1], 0.0])


def _reduced_newton(model, xn, y, act, red_nodes, tol, max_iter=60):
    """Newton on grad_{C'} g = 0 with the other nodes held (Eqn reduced system)."""
    free = model.free_nodes
    pos = -np.ones(model.mesh.n, dtype=np.int64)
    pos[free] = np.arange(free.size)
    rdofs = (red_nodes[:, None] * 3 + np.arange(3)).ravel()          # full-vector dofs
    fdofs = (pos[red_nodes][:, None] * 3 + np.arange(3)).ravel()     # positions in grad_g
    gr = model.grad_g(xn, y, act)[fdofs]
    ref = max(np.linalg.norm(gr), np.linalg.norm((model.m[:, None] * y / model.h ** 2)[red_nodes]))
    it = 0
    while np.linalg.norm(gr) > tol * ref and it < max_iter:
        H = model.hessian(xn, act)[rdofs][:, rdofs].tocsc()
        dx = spla.splu(H).solve(-gr)
        if not (np.all(np.isfinite(dx)) and dx @ gr < 0):
            dx = spla.splu(model.A_matrix()[rdofs][:, rdofs].tocsc()).solve(-gr)
        g0 = model.g_value(xn, y, act)
        slope = dx @ gr
        alpha = 1.0
        for _ in range(10):
            xt = np.array(xn, copy=True)
            xt[red_nodes] += alpha * dx.reshape(-1, 3)
            if model.g_value(xt, y, act) <= g0 + 1e-4 * alpha * slope + 1e-14 * abs(g0):
                break
            alpha *= 0.5
        xn = xt
        gr = model.grad_g(xn, y, act)[fdofs]
        it += 1
    return xn, it, float(np.linalg.norm(gr) / ref)


def step_complementarity(model, x, v, f_ext, cand, act=None, tol=1e-12, max_sets=64):
    """One implicit-Euler step with complementarity contact.  cand: node mask.
    Returns (x_next, v_next, info) with info['C'] (node ids, in the order they
    joined), info['rules'], info['xstar'] (c, 3)."""
    h = model.h
    y = model.predictor(x, v, f_ext)
    cand_nodes = np.flatnonzero(np.asarray(cand, dtype=bool) & ~model.dirichlet)
    C, rules = [], []
    for j in cand_nodes:
        if x[j, 2] <= 0.0:
            C.append(j), rules.append("drop")
        elif x[j, 2] + h * v[j, 2] <= 0.0:
            C.append(j), rules.append("ray")
    xn = np.array(y, copy=True)
    xn[model.dirichlet] = model.mesh.X[model.dirichlet]
    # tolerances of the set update: forces within rounding of zero do not release a
    # node, rounding-level penetrations do not add one (else the set can cycle)
    tau_r = 1e-8 * float(np.max(model.m)) * float(np.linalg.norm(model.gravity))
    tau_z = 1e-9 * model.mesh.dx
    # anti-cycling: with every coordinate of a node held, its normal force can be
    # negative while releasing it makes it penetrate; a node may leave once per
    # step -- if it penetrates afterwards it rejoins and stays ("locked")
    left, locked = set(), set()
    iters = 0
    for rounds in range(1, max_sets + 1):
        xs = np.array([contact_target(x[j], v[j], h, r) for j, r in zip(C, rules)]).reshape(-1, 3)
        xn[np.array(C, dtype=np.int64)] = xs
        red = np.setdiff1d(model.free_nodes, np.array(C, dtype=np.int64))
        xn, it, rel = _reduced_newton(model, xn, y, act, red, tol)
        iters += it
        r = (model.m[:, None] * (xn - y) / h ** 2 + model.grad_E(xn, act))
        leave = {j for j in C if r[j, 2] < -tau_r and j not in locked}
        inC = set(C)
        join = [j for j in cand_nodes if j not in inC and xn[j, 2] < -tau_z]
        if not leave and not join or rounds == max_sets:
            break
        locked |= {j for j in join if j in left}
        left |= leave
        keep = [(j, rl) for j, rl in zip(C, rules) if j not in leave]
        C = [j for j, _ in keep] + join
        rules = [rl for _, rl in keep] + ["drop"] * len(join)
    xs = np.array([contact_target(x[j], v[j], h, r) for j, r in zip(C, rules)]).reshape(-1, 3)
    info = {"C": np.array(C, dtype=np.int64), "rules": list(rules), "xstar": xs, "y": y, "iters": iters,
            "rounds": rounds, "residual": rel, "tau_r": tau_r, "tau_z": tau_z,
            "locked": np.array(sorted(locked), dtype=np.int64),
            "force": (model.m[:, None] * (xn - y) / h ** 2 + model.grad_E(xn, act))[np.array(C, dtype=np.int64)]}
    return xn, (xn - x) / h, info


def rollout_complementarity(model, x0, v0, f_ext, cand, T, act=None, tol=1e-12):
    xs, vs, infos = [np.array(x0, dtype=np.float64)], [np.array(v0, dtype=np.float64)], []
    for t in range(T):
        xn, vn, info = step_complementarity(model, xs[-1], vs[-1], f_ext, cand,
                                            None if act is None else act[t], tol)
        xs.append(xn), vs.append(vn), infos.append(info)
    return np.stack(xs), np.stack(vs), infos


def target_vjp(xt, vt, h, rule, g):
    """(dL/dx_t, dL/dv_t) of one node from dL/dx* = g through contact_target."""
    if rule == "ray":
        s = xt[2] / (-vt[2])
        w = -(g[0] * vt[0] + g[1] * vt[1]) / vt[2]   # d s / d z_t = -1/v_z, d s / d v_z = -s/v_z
        return np.array([g[0], g[1], w]), np.array([s * g[0], s * g[1], s * w])
    return np.array([g[0], g[1], 0.0]), np.zeros(3)


def backward_complementarity(model, xs, vs, infos, gx, gv=None, act=None):
    """Back-propagation through a rollout with complementarity contact (Alg. 5,
    solved directly): per step, with the final contact set C of that step,
      (Hess g)_{C'C'} z_{C'} = gbar_{C'},  z_C = 0,
      dL/dy = M z / h^2,  dL/dx* = gbar_C - (Hess g)_{C C'} z_{C'},
    then x* -> (x_t, v_t) through contact_target.  Returns g_x0, g_v0, g_wc, g_wv."""
    T = xs.shape[0] - 1
    n = model.mesh.n
    h = model.h
    free = model.free_nodes
    Vq = model.mesh.Vq
    ax = np.array(gx[T], dtype=np.float64, copy=True)
    av = np.zeros((n, 3)) if gv is None else np.array(gv[T], dtype=np.float64, copy=True)
    g_wc = np.zeros(model.mesh.e)
    g_wv = np.zeros(model.mesh.e)
    for t in reversed(range(T)):
        a_t = None if act is None else act[t]
        C = infos[t]["C"]
        red = np.setdiff1d(free, C)
        gbar = ax + av / h
        Hf = model.hessian(xs[t + 1], a_t)
        rd = (red[:, None] * 3 + np.arange(3)).ravel()
        z = np.zeros((n, 3))
        if red.size:
            z[red] = spla.splu(Hf[rd][:, rd].tocsc()).solve(gbar[red].ravel()).reshape(-1, 3)
        dLdy = model.m[:, None] * z / h ** 2
        new_ax = np.zeros((n, 3))
        new_av = np.zeros((n, 3))
        new_ax[free] = (dLdy - av / h)[free]
        new_av[free] = (h * dLdy)[free]
        if C.size:
            Hz = (Hf @ z.ravel()).reshape(-1, 3)
            gstar = gbar[C] - Hz[C]
            for k, j in enumerate(C):
                dx, dv = target_vjp(xs[t][j], vs[t][j], h, infos[t]["rules"][k], gstar[k])
                new_ax[j] += dx
                new_av[j] += dv
        loc = model.local(xs[t + 1], a_t)
        Gz = model.mesh.deformation_gradients(z)
        if "R" in loc:
            g_wc += -Vq * np.einsum("eqij,eqij->e", Gz, loc["F"] - loc["R"])
        if "D" in loc:
            g_wv += -Vq * np.einsum("eqij,eqij->e", Gz, loc["F"] - loc["D"])
        ax = new_ax + gx[t]
        av = new_av + (0.0 if gv is None else gv[t])
    return {"g_x0": ax, "g_v0": av, "g_wc": g_wc, "g_wv": g_wv}
