"""Pins for the projections (supplement energy definitions): library polar
decomposition, manifold membership, idempotence, rotation equivariance,
brute-force minimality, and central finite differences for every Jacobian."""
import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

from oracle import projections as pj


def _randF(rng, n, scale=0.3):
    F = np.eye(3)[None] + scale * rng.standard_normal((n, 3, 3))
    F[np.linalg.det(F) <= 0.05] = np.eye(3)
    return F


def _rot(rng):
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    return Q


def test_corotated_matches_scipy_polar():
    rng = np.random.default_rng(0)
    F = _randF(rng, 200)
    R = pj.project_corotated(F)
    for k in range(F.shape[0]):
        u, p = scipy.linalg.polar(F[k])
        assert np.allclose(R[k], u, atol=1e-12)


def test_corotated_manifold_idempotent_equivariant():
    rng = np.random.default_rng(1)
    F = _randF(rng, 100)
    R = pj.project_corotated(F)
    assert np.allclose(np.einsum("nki,nkj->nij", R, R), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-12)
    assert np.allclose(pj.project_corotated(R), R, atol=1e-12)
    Q = _rot(rng)
    assert np.allclose(pj.project_corotated(Q[None] @ F), Q[None] @ R, atol=1e-12)


def test_signed_svd_inverted():
    F = np.diag([2.0, 1.0, -0.5])
    U, s, V = pj.signed_svd(F)
    assert np.isclose(np.linalg.det(U), 1) and np.isclose(np.linalg.det(V), 1)
    assert s[2] < 0 and np.allclose(U @ np.diag(s) @ V.T, F)


def test_volume_projection_properties():
    rng = np.random.default_rng(2)
    F = _randF(rng, 100)
    D = pj.project_volume(F)
    assert np.allclose(np.linalg.det(D), 1.0, atol=1e-12)
    assert np.allclose(pj.project_volume(D), D, atol=1e-12)
    # det F = 1 is already on the manifold
    G = F / np.cbrt(np.linalg.det(F))[:, None, None]
    assert np.allclose(pj.project_volume(G), G, atol=1e-11)


def test_volume_projection_minimal_vs_brute_force():
    rng = np.random.default_rng(3)
    F = _randF(rng, 6, scale=0.25)
    D = pj.project_volume(F)
    for k in range(F.shape[0]):
        best = np.inf
        for _ in range(20):
            x0 = (np.eye(3) + 0.3 * rng.standard_normal((3, 3))).ravel()
            res = scipy.optimize.minimize(
                lambda d: np.sum((d - F[k].ravel()) ** 2), x0,
                constraints=[{"type": "eq", "fun": lambda d: np.linalg.det(d.reshape(3, 3)) - 1.0}],
                method="SLSQP", options={"ftol": 1e-14, "maxiter": 500})
            if res.success:
                best = min(best, res.fun)
        assert np.sum((D[k] - F[k]) ** 2) <= best + 1e-9


def _fd_jac(P, F, eps=1e-6):
    J = np.zeros((9, 9))
    for c in range(9):
        d = np.zeros(9)
        d[c] = eps
        J[:, c] = (P(F + d.reshape(3, 3)) - P(F - d.reshape(3, 3))).ravel() / (2 * eps)
    return J


@pytest.mark.parametrize("kind", ["corotated", "volume"])
def test_isotropic_jacobians_fd_and_symmetric(kind):
    rng = np.random.default_rng(4)
    F = _randF(rng, 30)
    proj = pj.project_corotated if kind == "corotated" else pj.project_volume
    jac = pj.jacobian_corotated if kind == "corotated" else pj.jacobian_volume
    Jb = jac(F)
    for k in range(F.shape[0]):
        Jfd = _fd_jac(lambda G: proj(G[None])[0], F[k])
        assert np.max(np.abs(Jb[k] - Jfd)) <= 1e-7 * max(1.0, np.max(np.abs(Jfd)))
        assert np.allclose(Jb[k], Jb[k].T, atol=1e-10)


@pytest.mark.parametrize("kind", ["corotated", "volume"])
def test_jacobian_at_repeated_singular_values(kind):
    """Rest state F = I and F = diag(a, a, b): divided differences hit their limit."""
    proj = pj.project_corotated if kind == "corotated" else pj.project_volume
    jac = pj.jacobian_corotated if kind == "corotated" else pj.jacobian_volume
    for F in (np.eye(3), np.diag([1.1, 1.1, 0.9]), np.diag([1.2, 0.95, 0.95])):
        Jfd = _fd_jac(lambda G: proj(G[None])[0], F)
        assert np.max(np.abs(jac(F) - Jfd)) < 1e-7


def test_corotated_jacobian_at_identity_is_skew_projector():
    J = pj.jacobian_corotated(np.eye(3))
    # dR at F = I is the skew part of dF
    rng = np.random.default_rng(5)
    dF = rng.standard_normal((3, 3))
    assert np.allclose((J @ dF.ravel()).reshape(3, 3), 0.5 * (dF - dF.T), atol=1e-14)


def test_muscle_projection_and_jacobian():
    rng = np.random.default_rng(6)
    f = rng.standard_normal(3)
    a = 0.2
    p = pj.project_muscle(f, a)
    assert np.isclose(np.linalg.norm(p), 1 - a)
    assert np.allclose(pj.project_muscle(p, a), p)
    J = pj.jacobian_muscle(f, a)
    eps = 1e-6
    Jfd = np.stack([(pj.project_muscle(f + eps * e, a) - pj.project_muscle(f - eps * e, a)) / (2 * eps)
                    for e in np.eye(3)], axis=1)
    assert np.allclose(J, Jfd, atol=1e-8)


def test_ground_projection():
    x = np.array([[0.1, 0.2, -0.3], [0.0, 0.0, 0.4], [1.0, 1.0, 0.0]])
    p = pj.project_ground(x)
    assert np.all(p[:, 2] >= 0) and np.allclose(pj.project_ground(p), p)
    assert np.allclose(p[:, :2], x[:, :2])
