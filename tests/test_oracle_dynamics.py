"""Pins for the oracle's forward step and adjoint (Sec. 3, Sec. 4, Sec. 5.1):
rest / translation / rotation invariants, linear momentum, the PD fixed point
equals the Newton fixed point, a closed-form static contact balance, central
finite differences of every gradient block, the adjoint against a
finite-difference linearisation of one step, the large-mesh MINRES adjoint
against a dense solve, a forward-mode / reverse-mode dot-product test, and the
spectral radius of A^-1 Delta A (Sec. 6 ablation)."""
import dataclasses

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import adjoint, newton, pd_cpu
from oracle.model import Model
from workloads import Scene, cantilever_c1, small_beam


def _rot(rng):
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    return Q


def _free_scene(sc, **kw):
    n = sc.x0.shape[0]
    base = dict(dirichlet=np.zeros(n, dtype=np.uint8), gravity=np.zeros(3),
                f_ext=np.zeros((n, 3)))
    base.update(kw)
    return dataclasses.replace(sc, **base)


def test_rest_state_stays_at_rest():
    sc = dataclasses.replace(cantilever_c1(T=3), gravity=np.zeros(3))
    sc.v0[:] = 0.0
    m = Model(sc)
    xs, vs, _ = newton.rollout(m, sc.x0, sc.v0, sc.f_ext)
    assert np.max(np.abs(xs - sc.x0[None])) < 1e-14
    assert np.max(np.abs(vs)) < 1e-12


def test_uniform_translation_exact():
    sc = _free_scene(small_beam(3, 2, 2, T=4))
    u = np.array([0.3, -0.1, 0.2])
    sc.v0[:] = u
    m = Model(sc)
    xs, vs, _ = newton.rollout(m, sc.x0, sc.v0, sc.f_ext)
    for t in range(xs.shape[0]):
        assert np.allclose(xs[t], sc.x0 + t * sc.h * u, atol=1e-13, rtol=0)


def test_rigidly_rotated_rest_mesh_stays():
    rng = np.random.default_rng(0)
    Q = _rot(rng)
    sc = _free_scene(small_beam(3, 2, 2, T=2))
    x0 = sc.x0 @ Q.T + np.array([0.1, 0.2, 0.3])
    sc.v0[:] = 0.0
    m = Model(sc)
    xs, _, _ = newton.rollout(m, x0, sc.v0, sc.f_ext)
    assert np.max(np.abs(xs[-1] - x0)) < 1e-13


def test_linear_momentum_conserved():
    sc = _free_scene(small_beam(3, 2, 2, T=5))
    rng = np.random.default_rng(1)
    v0 = 0.05 * rng.standard_normal(sc.x0.shape)
    m = Model(sc)
    xs, vs, _ = newton.rollout(m, sc.x0, v0, sc.f_ext)
    p0 = (m.m[:, None] * v0).sum(0)
    for t in range(1, xs.shape[0]):
        assert np.allclose((m.m[:, None] * vs[t]).sum(0), p0, atol=1e-12)


def test_newton_residual_and_pd_same_fixed_point():
    sc = cantilever_c1(T=4)
    m = Model(sc)
    xs, _, infos = newton.rollout(m, sc.x0, sc.v0, sc.f_ext)
    for info in infos:
        assert info["residual"] <= 1e-12 * info["ref"]
    xp, _, pinfo = pd_cpu.rollout(m, sc.x0, sc.v0, sc.f_ext)
    assert np.max(np.abs(xp - xs)) < 1e-10
    assert all(i["iters"] > 1 for i in pinfo)


def test_static_contact_force_balances_weight():
    """A cube resting on the ground: at static equilibrium the penalty forces
    sum to the total weight (force balance, exact for any distribution)."""
    N = 2
    from workloads import contact_cube_c3
    sc = contact_cube_c3(N=N, T=1)
    sc = dataclasses.replace(sc, origin=np.array([0.0, 0.0, 0.0]), h=0.05, mu=0.0)
    sc.x0[:, 2] -= 0.05
    sc.v0[:] = 0.0
    m = Model(sc)
    x, v = sc.x0, sc.v0
    for _ in range(150):
        x, v, _ = newton.newton_step(m, x, v, sc.f_ext)
    z = x[m.contact, 2]
    Fc = np.sum(m.k * np.maximum(-z, 0.0))
    W = m.m.sum() * 9.81
    assert abs(Fc - W) < 1e-6 * W
    assert np.max(np.abs(v)) < 1e-6


def tiny_everything_scene(T=3):
    """2x1x2 cells with volume + muscle energies, ground contact and friction.

    Heavy (rho = 1e4) soft material so that the PD splitting converges in a
    few hundred iterations: near-rigid rotations contract by about
    1 - (m/h^2)/(E dx) per plain PD iteration."""
    nx, ny, nz = 2, 1, 2
    n = (nx + 1) * (ny + 1) * (nz + 1)
    e = nx * ny * nz
    rng = np.random.default_rng(11)
    ids = np.arange(n)
    k = ids % (nz + 1)
    j = (ids // (nz + 1)) % (ny + 1)
    i = ids // ((nz + 1) * (ny + 1))
    x0 = np.stack([i, j, k], 1) * 0.01 + np.array([0.0, 0.0, -2e-6])
    x0 = x0 + 1e-4 * rng.standard_normal(x0.shape) * np.array([1, 1, 0])
    v0 = 0.05 * rng.standard_normal((n, 3))
    fib = rng.standard_normal((e, 3))
    fib /= np.linalg.norm(fib, axis=1, keepdims=True)
    return Scene(name="tiny", nx=nx, ny=ny, nz=nz, dx=0.01, origin=np.zeros(3), cell_mask=None,
                 density=1e4, youngs=1e5 * np.exp(0.2 * rng.standard_normal(e)), poisson=0.4,
                 corotated=True, volume=True, muscle=np.ones(e, dtype=np.uint8), fiber=fib,
                 dirichlet=np.zeros(n, dtype=np.uint8), contact=(k == 0).astype(np.uint8),
                 gravity=np.array([0.0, 0.0, -9.81]), h=0.01, T=T, x0=x0, v0=v0,
                 f_ext=0.01 * rng.standard_normal((n, 3)),
                 act=rng.uniform(0, 0.3, size=(T, e)), k_contact=1e3, mu=0.5,
                 loss_w=rng.standard_normal((n, 3)), tol_fwd=1e-12, tol_bwd=1e-12)


def _loss(sc, **over):
    m = Model(sc, youngs=over.get("youngs"), poisson=over.get("poisson"), mu=over.get("mu"))
    xs, _, _ = newton.rollout(m, over.get("x0", sc.x0), over.get("v0", sc.v0),
                              over.get("f_ext", sc.f_ext), over.get("act", sc.act), mu=over.get("mu"))
    return float(np.sum(sc.loss_w * xs[-1]))


def test_gradients_match_central_fd_everything():
    sc = tiny_everything_scene()
    m = Model(sc)
    xs, vs, _ = newton.rollout(m, sc.x0, sc.v0, sc.f_ext, sc.act)
    # contact must be active and both friction regimes visited for this to pin anything
    assert np.any(xs[:-1][:, m.contact, 2] < 0)
    _, gx = adjoint.final_position_loss(m, xs, sc.loss_w)
    g = adjoint.backward(m, xs, vs, gx, act=sc.act)
    gE, gnu = adjoint.material_gradients(m, g)
    rng = np.random.default_rng(3)

    def fd(fun, eps):
        return (fun(eps) - fun(-eps)) / (2 * eps)

    checks = []
    d = rng.standard_normal(sc.x0.shape)
    checks.append((fd(lambda s: _loss(sc, x0=sc.x0 + s * d), 1e-7), np.sum(g["g_x0"] * d)))
    checks.append((fd(lambda s: _loss(sc, v0=sc.v0 + s * d), 1e-6), np.sum(g["g_v0"] * d)))
    # small step: a node sits ~1.7e-5 from the static/dynamic friction switch
    checks.append((fd(lambda s: _loss(sc, f_ext=sc.f_ext + s * d), 1e-6), np.sum(g["g_fext"] * d)))
    dE = rng.standard_normal(m.mesh.e) * sc.youngs
    checks.append((fd(lambda s: _loss(sc, youngs=sc.youngs + s * dE), 1e-6), np.sum(gE * dE)))
    checks.append((fd(lambda s: _loss(sc, poisson=sc.poisson + s), 1e-6), gnu))
    checks.append((fd(lambda s: _loss(sc, mu=sc.mu + s), 1e-6), g["g_mu"]))
    da = rng.standard_normal(sc.act.shape)
    checks.append((fd(lambda s: _loss(sc, act=sc.act + s * da), 1e-6), np.sum(g["g_act"] * da)))
    for num, ana in checks:
        assert abs(num - ana) <= 2e-6 * max(abs(num), 1e-12), (num, ana)


def test_adjoint_matches_fd_linearisation_of_one_step():
    """<gbar, dx/dy dy> = <M z / h^2, dy> (Eqns 10-12) with dx/dy dy by FD."""
    sc = cantilever_c1(T=1)
    m = Model(sc)
    xs, vs, infos = newton.rollout(m, sc.x0, sc.v0, sc.f_ext)
    rng = np.random.default_rng(4)
    gbar = rng.standard_normal(xs[1].shape)
    gbar[m.dirichlet] = 0
    dy = rng.standard_normal(xs[1].shape)
    dy[m.dirichlet] = 0
    # a velocity perturbation dv moves y by h dv
    eps = 1e-6

    def x_of(s):
        x, _, _ = newton.newton_step(m, sc.x0, sc.v0 + s * dy / m.h, sc.f_ext)
        return x
    jdy = (x_of(eps) - x_of(-eps)) / (2 * eps)
    H = m.hessian(xs[1])[m.free_dofs][:, m.free_dofs].tocsc()
    z = np.zeros_like(gbar)
    z[m.free_nodes] = spla.spsolve(H, gbar[m.free_nodes].ravel()).reshape(-1, 3)
    lhs = np.sum(gbar * jdy)
    rhs = np.sum(m.m[:, None] * z / m.h ** 2 * dy)
    assert abs(lhs - rhs) < 1e-7 * abs(rhs)


def test_spectral_radius_below_one_on_cantilever():
    sc = cantilever_c1(T=10)
    m = Model(sc)
    xs, _, _ = newton.rollout(m, sc.x0, sc.v0, sc.f_ext)
    dofs = m.free_dofs
    A = m.A_matrix()[dofs][:, dofs].toarray()
    H = m.hessian(xs[-1])[dofs][:, dofs].toarray()
    rho = np.max(np.abs(np.linalg.eigvals(np.linalg.solve(A, A - H))))
    assert 0.0 < rho < 1.0


def test_minres_adjoint_matches_dense_solve():
    """The large-mesh oracle adjoint (A^-1-preconditioned MINRES on Hess g z = gbar,
    Sec. 4 Eqn 10) agrees with a dense direct solve of the same system on the
    cantilever (600 free DoFs) at three successive states."""
    sc = cantilever_c1(T=3)
    m = Model(sc)
    xs, _, _ = newton.rollout(m, sc.x0, sc.v0, sc.f_ext)
    Afac = pd_cpu.ScalarA(m)
    dofs = m.free_dofs
    rng = np.random.default_rng(11)
    for t in range(3):
        gbar = rng.standard_normal(dofs.size)
        z = pd_cpu.adjoint_solve_minres(m, Afac, xs[t + 1], gbar)
        Hd = m.hessian(xs[t + 1])[dofs][:, dofs].toarray()
        zd = np.linalg.solve(Hd, gbar)
        assert np.linalg.norm(z - zd) <= 1e-9 * np.linalg.norm(zd)


def test_dot_product_forward_vs_reverse_mode():
    """<gbar, J dv> = <J^T gbar, dv> for one step: J dv from the forward-mode
    linearisation Hess g dx = M dy / h^2 with dy = h dv (dense solve), J^T gbar from
    the oracle's reverse pass (dL/dv_0 = h M z / h^2, Eqns 10-12)."""
    sc = cantilever_c1(T=1)
    m = Model(sc)
    xs, vs, _ = newton.rollout(m, sc.x0, sc.v0, sc.f_ext)
    rng = np.random.default_rng(12)
    n = xs.shape[1]
    gbar = rng.standard_normal((n, 3))
    gbar[m.dirichlet] = 0.0
    dv = rng.standard_normal((n, 3))
    dv[m.dirichlet] = 0.0
    dofs = m.free_dofs
    Hd = m.hessian(xs[1])[dofs][:, dofs].toarray()
    rhs = (m.m[:, None] * (m.h * dv) / m.h ** 2)[m.free_nodes].ravel()
    dx = np.zeros((n, 3))
    dx[m.free_nodes] = np.linalg.solve(Hd, rhs).reshape(-1, 3)
    gx = np.zeros_like(xs)
    gx[1] = gbar
    g = adjoint.backward(m, xs, vs, gx)
    lhs = np.sum(gbar * dx)
    rhs_rev = np.sum(g["g_v0"] * dv)
    assert abs(lhs - rhs_rev) <= 1e-12 * max(abs(lhs), 1e-300) + 1e-300, (lhs, rhs_rev)
