"""Pins for the oracle's Neo-Hookean material (Sec. 8; the paper names the model
without printing it, reading in oracle/neohookean.py): the stress against central
differences of the energy density, the tangent against central differences of the
stress, frame indifference and a stress-free rest state, the small-strain limit
(linear elasticity with the same Lame parameters, a textbook closed form), the
mesh gradient and Hessian against differences of the energy and gradient, the PD +
L-BFGS fixed point (A as initial Hessian) against Newton's, and the adjoint
gradients against central differences of a rollout loss."""
import dataclasses

import numpy as np

from oracle import adjoint, neohookean as nh, newton, pd_cpu
from oracle.model import Model
from workloads import neohookean_beam

MU, LAM = 3.4e4, 3.1e5


def _rot(rng):
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    return Q


def _F(rng, scale):
    F = np.eye(3) + scale * rng.standard_normal((3, 3))
    assert np.linalg.det(F) > 0.2
    return F


def test_stress_is_energy_derivative():
    rng = np.random.default_rng(1)
    for scale in (1e-3, 0.1, 0.3):
        F = _F(rng, scale)
        P = nh.first_piola(F, MU, LAM)
        eps = 1e-6
        for i in range(3):
            for j in range(3):
                E = np.zeros((3, 3))
                E[i, j] = eps
                fd = (nh.energy_density(F + E, MU, LAM) - nh.energy_density(F - E, MU, LAM)) / (2 * eps)
                assert abs(fd - P[i, j]) <= 1e-6 * np.abs(P).max() + 1e-6, (scale, i, j)


def test_tangent_is_stress_derivative():
    rng = np.random.default_rng(2)
    for scale in (0.05, 0.3):
        F = _F(rng, scale)
        T = nh.tangent(F, MU, LAM)
        eps = 1e-6
        for k in range(9):
            E = np.zeros((3, 3))
            E[k // 3, k % 3] = eps
            fd = (nh.first_piola(F + E, MU, LAM) - nh.first_piola(F - E, MU, LAM)).ravel() / (2 * eps)
            assert np.abs(fd - T[:, k]).max() <= 1e-6 * np.abs(T).max()
        # the tangent is symmetric (second derivative of an energy)
        assert np.abs(T - T.T).max() <= 1e-9 * np.abs(T).max()


def test_rest_state_and_frame_indifference():
    rng = np.random.default_rng(3)
    for _ in range(5):
        R = _rot(rng)
        assert abs(nh.energy_density(R, MU, LAM)) <= 1e-9 * MU
        assert np.abs(nh.first_piola(R, MU, LAM)).max() <= 1e-9 * MU
        F = _F(rng, 0.2)
        assert abs(nh.energy_density(R @ F, MU, LAM) - nh.energy_density(F, MU, LAM)) <= 1e-9 * MU
        assert np.abs(nh.first_piola(R @ F, MU, LAM) - R @ nh.first_piola(F, MU, LAM)).max() <= 1e-8 * MU


def test_small_strain_limit_is_linear_elasticity():
    """P(I + e H) / e -> mu (H + H^T) + lam tr(H) I and psi / e^2 -> mu |sym H|^2 + lam/2 tr(H)^2."""
    rng = np.random.default_rng(4)
    H = rng.standard_normal((3, 3))
    lin_P = MU * (H + H.T) + LAM * np.trace(H) * np.eye(3)
    S = 0.5 * (H + H.T)
    lin_psi = MU * np.sum(S * S) + 0.5 * LAM * np.trace(H) ** 2
    for e in (1e-3, 1e-4):
        P = nh.first_piola(np.eye(3) + e * H, MU, LAM) / e
        psi = nh.energy_density(np.eye(3) + e * H, MU, LAM) / e ** 2
        assert np.abs(P - lin_P).max() <= 20 * e * np.abs(lin_P).max()
        assert abs(psi - lin_psi) <= 20 * e * abs(lin_psi)


def _deformed(sc, rng, scale=0.05):
    return sc.x0 + scale * sc.dx * rng.standard_normal(sc.x0.shape)


def test_mesh_gradient_and_hessian_match_differences():
    sc = neohookean_beam(4, 2, 3, T=1)
    m = Model(sc)
    rng = np.random.default_rng(5)
    x = _deformed(sc, rng, 0.3)
    g = m.grad_E(x)
    d = rng.standard_normal(x.shape)
    eps = 1e-7
    fd = (m.energy(x + eps * d) - m.energy(x - eps * d)) / (2 * eps)
    assert abs(fd - np.sum(g * d)) <= 1e-6 * abs(fd)
    H = m.hessian(x)
    Hd = (H @ d.ravel()).reshape(x.shape) - (m.m / m.h ** 2)[:, None] * d
    fdg = (m.grad_E(x + eps * d) - m.grad_E(x - eps * d)) / (2 * eps)
    assert np.abs(fdg - Hd).max() <= 1e-6 * np.abs(Hd).max()


def test_pd_lbfgs_reaches_the_newton_fixed_point():
    """Quasi-Newton with the PD matrix A as initial Hessian (the paper's route for
    non-PD materials) converges to Newton's implicit-Euler step."""
    sc = neohookean_beam(5, 3, 4, T=1, twist=20.0)
    m = Model(sc)
    xn, _, _ = newton.newton_step(m, sc.x0, sc.v0, sc.f_ext)
    xp, _, info = pd_cpu.pd_lbfgs_step(m, pd_cpu.ScalarA(m), sc.x0, sc.v0, sc.f_ext, None, None, 1e-12, 5, 5000)
    assert np.linalg.norm(xp - xn) <= 1e-9 * np.linalg.norm(xn - sc.x0)


def _loss(sc, **over):
    m = Model(sc, youngs=over.get("youngs"), poisson=over.get("poisson"))
    xs, _, _ = newton.rollout(m, sc.x0, over.get("v0", sc.v0), over.get("f_ext", sc.f_ext))
    return float(np.sum(sc.loss_w * xs[-1]))


def test_adjoint_matches_central_differences():
    sc = neohookean_beam(4, 2, 3, T=3, twist=15.0)
    m = Model(sc)
    xs, vs, _ = newton.rollout(m, sc.x0, sc.v0, sc.f_ext)
    _, gx = adjoint.final_position_loss(m, xs, sc.loss_w)
    g = adjoint.backward(m, xs, vs, gx)
    gE, gnu = adjoint.material_gradients(m, g)
    rng = np.random.default_rng(6)

    def fd(fun, eps):
        return (fun(eps) - fun(-eps)) / (2 * eps)
    d = rng.standard_normal(sc.x0.shape)
    d[m.dirichlet] = 0.0
    checks = [(fd(lambda s: _loss(sc, v0=sc.v0 + s * d), 1e-6), np.sum(g["g_v0"] * d)),
              (fd(lambda s: _loss(sc, f_ext=sc.f_ext + s * d), 1e-6), np.sum(g["g_fext"] * d))]
    dE = rng.standard_normal(m.mesh.e) * sc.youngs
    checks.append((fd(lambda s: _loss(sc, youngs=sc.youngs + s * dE), 1e-6), np.sum(gE * dE)))
    checks.append((fd(lambda s: _loss(sc, poisson=sc.poisson + s), 1e-6), gnu))
    for num, ana in checks:
        assert abs(num - ana) <= 2e-6 * max(abs(num), 1e-12), (num, ana)


def test_neohookean_differs_from_corotated_at_large_strain():
    """The material is actually switched: at a large rotation-free stretch the
    Neo-Hookean and the corotated + volume energies differ."""
    sc = neohookean_beam(4, 2, 3, T=1)
    x = sc.x0 * np.array([1.3, 1.0, 1.0])
    e_nh = Model(sc).energy(x)
    e_pd = Model(dataclasses.replace(sc, neohookean=False)).energy(x)
    assert abs(e_nh - e_pd) > 0.05 * abs(e_pd)
