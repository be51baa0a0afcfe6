"""Writes the stored oracle results used by the GPU parity tests.

Only oracle/ and workloads/ are called: every stored value comes from the FP64
CPU oracle (Newton forward, direct adjoint), never from the CUDA path.
Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import adjoint, newton, pd_cpu  # noqa: E402
from oracle.model import Model  # noqa: E402
from workloads import beam_c2, cantilever_c1  # noqa: E402


def c1():
    sc = cantilever_c1()
    model = Model(sc)
    xs, vs, infos = newton.rollout(model, sc.x0, sc.v0, sc.f_ext)
    loss, gx = adjoint.final_position_loss(model, xs, sc.loss_w)
    g = adjoint.backward(model, xs, vs, gx)
    gE, gnu = adjoint.material_gradients(model, g)
    np.savez_compressed(os.path.join(HERE, "c1_cantilever_oracle.npz"), xs=xs, vs=vs, loss=loss,
                        g_v0=g["g_v0"], g_x0=g["g_x0"], g_wc=g["g_wc"], g_E=gE, g_nu=gnu,
                        newton_iters=np.array([i["iters"] for i in infos]))


def c2(T=2, n_sample=2000):
    """32x32x64 beam, first T steps: oracle PD + L-BFGS forward polished to
    |grad g| <= 1e-12 (same fixed point as Newton, Sec. 3) and the
    A^-1-preconditioned MINRES adjoint to 1e-12; stores sampled nodes/elements."""
    sc = beam_c2(T=T)
    model = Model(sc)
    Afac = pd_cpu.ScalarA(model)
    xs = [sc.x0.copy()]
    vs = [sc.v0.copy()]
    for t in range(T):
        xn, vn, info = pd_cpu.pd_lbfgs_step(model, Afac, xs[-1], vs[-1], sc.f_ext, None, None, 1e-12, 5, 5000)
        print("step", t, info, flush=True)
        xs.append(xn)
        vs.append(vn)
    xs = np.stack(xs)
    vs = np.stack(vs)
    # adjoint by MINRES (full linearisation) per step, reverse
    n = model.mesh.n
    h = model.h
    ax = np.array(sc.loss_w, dtype=np.float64)
    av = np.zeros((n, 3))
    gE_wc = np.zeros(model.mesh.e)
    gE_wv = np.zeros(model.mesh.e)
    Vq = model.mesh.Vq
    for t in reversed(range(T)):
        gbar = (ax + av / h)[model.free_nodes].ravel()
        zf = pd_cpu.adjoint_solve_minres(model, Afac, xs[t + 1], gbar, None, 1e-12)
        z = np.zeros((n, 3))
        z[model.free_nodes] = zf.reshape(-1, 3)
        dLdy = model.m[:, None] * z / h ** 2
        new_ax = np.zeros((n, 3))
        new_av = np.zeros((n, 3))
        new_ax[model.free_nodes] = (dLdy - av / h)[model.free_nodes]
        new_av[model.free_nodes] = (h * dLdy)[model.free_nodes]
        loc = model.local(xs[t + 1])
        Gz = model.mesh.deformation_gradients(z)
        gE_wc += -Vq * np.einsum("eqij,eqij->e", Gz, loc["F"] - loc["R"])
        gE_wv += -Vq * np.einsum("eqij,eqij->e", Gz, loc["F"] - loc["D"])
        ax, av = new_ax, new_av
        print("adjoint step", t, flush=True)
    rng = np.random.default_rng(2025)
    nodes = np.sort(rng.choice(n, size=n_sample, replace=False))
    cells = np.sort(rng.choice(model.mesh.e, size=n_sample, replace=False))
    np.savez_compressed(os.path.join(HERE, "c2_beam_T%d_oracle_sampled.npz" % T), T=T, nodes=nodes, cells=cells,
                        xs=xs[:, nodes], x_norm=np.linalg.norm(xs.reshape(T + 1, -1), axis=1),
                        g_v0=av[nodes], g_v0_norm=np.linalg.norm(av), g_wc=gE_wc[cells], g_wv=gE_wv[cells],
                        g_wc_norm=np.linalg.norm(gE_wc), g_wv_norm=np.linalg.norm(gE_wv),
                        loss=float(np.sum(sc.loss_w * xs[-1])))


def c3(T=2, n_sample=2000):
    """24^3 contact cube (penalty ground contact and friction, Sec. 5.1), first T
    steps: Newton forward and the full-linearisation adjoint (direct solves);
    stores sampled nodes with full-vector norms, the friction-coefficient gradient
    and the loss sum(w x_T)."""
    from workloads import contact_cube_c3
    sc = contact_cube_c3(T=T)
    model = Model(sc)
    xs, vs, infos = newton.rollout(model, sc.x0, sc.v0, sc.f_ext, mu=sc.mu, T=T)
    for t, i in enumerate(infos):
        print("step", t, i, flush=True)
    loss, gx = adjoint.final_position_loss(model, xs, sc.loss_w)
    g = adjoint.backward(model, xs, vs, gx, mu=sc.mu)
    n = xs.shape[1]
    rng = np.random.default_rng(2026)
    nodes = np.sort(rng.choice(n, size=min(n_sample, n), replace=False))
    np.savez_compressed(os.path.join(HERE, "c3_cube_T%d_oracle_sampled.npz" % T), T=T, nodes=nodes,
                        xs=xs[:, nodes], x_norm=np.linalg.norm(xs.reshape(T + 1, -1), axis=1),
                        g_v0=g["g_v0"][nodes], g_v0_norm=np.linalg.norm(g["g_v0"]),
                        g_x0=g["g_x0"][nodes], g_x0_norm=np.linalg.norm(g["g_x0"]),
                        g_mu=np.asarray(g["g_mu"]), loss=loss,
                        contact_nodes=np.array([int(np.sum((xs[t][:, 2] < 0) & (sc.contact > 0)))
                                                for t in range(T + 1)]))


if __name__ == "__main__":
    which = sys.argv[1:] or ["c1"]
    if "c1" in which:
        c1()
    if "c2" in which:
        c2()
    if "c2_10" in which:
        c2(T=10)   # a longer prefix of the 100-step benchmark horizon
    if "c3" in which:
        c3()
    if "c3_24" in which:
        c3(T=24)   # the cube reaches the ground near step 20: contact and friction engage
    print("written")
