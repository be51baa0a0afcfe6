"""Projections onto the PD constraint manifolds and their Jacobians
(oracle; test infrastructure only).

Sec. 3 (Eqn 16): E_c(x) = min_{p in M_c} w_c/2 |G_c x - p|^2; the local step
projects G_c x onto M_c.  Sec. 4 (Eqn 21) needs dp_c/dx for Delta A.

  corotated  M = SO(3): p = R, the rotation of the polar decomposition of F
             (supplement, "Background elasticity").
  volume     M = {det D = 1}: with F = U S V^T, D = U (S + d*) V^T where
             d* = argmin |d|^2 s.t. prod_i (S_ii + d_i) = 1 (supplement).
  muscle     project f = F m onto the sphere |p| = 1 - a (supplement,
             "Muscle fibers"; reading: the printed energy is garbled, the
             projection target radius is taken as 1 - a, a = contraction).
  contact    ground z = 0: p = (x, y, max(z, 0)) (Sec. 5.1, the obstacle
             surface and its exterior).

Jacobians of the isotropic projections use the derivative of a spectral
matrix function: with M = U^T dF V,
   (U^T dP V)_ii = sum_j ds_i/dsigma_j M_jj
   (U^T dP V)_ij = (s_i - s_j)/(sigma_i - sigma_j) sym(M)_ij
                 + (s_i + s_j)/(sigma_i + sigma_j) skew(M)_ij      (i != j)
For the volume projection ds/dsigma = I + dd*/dsigma comes from the KKT
sensitivity system of the supplement (Eqn S5).
"""
from __future__ import annotations

import numpy as np


def signed_svd(F: np.ndarray):
    """F = U diag(s) V^T with U, V proper rotations; s sorted by |s|
    descending, the last entry negative iff det F < 0.  Batched over leading
    axes.  Built on numpy.linalg.svd (LAPACK)."""
    U, s, Vt = np.linalg.svd(F)
    s = s.copy()
    U = U.copy()
    Vt = Vt.copy()
    du = np.linalg.det(U) < 0
    U[..., :, 2] = np.where(du[..., None], -U[..., :, 2], U[..., :, 2])
    s[..., 2] = np.where(du, -s[..., 2], s[..., 2])
    dv = np.linalg.det(Vt) < 0
    Vt[..., 2, :] = np.where(dv[..., None], -Vt[..., 2, :], Vt[..., 2, :])
    s[..., 2] = np.where(dv, -s[..., 2], s[..., 2])
    return U, s, np.swapaxes(Vt, -1, -2)


def project_corotated(F: np.ndarray) -> np.ndarray:
    U, _, V = signed_svd(F)
    return U @ np.swapaxes(V, -1, -2)


def volume_singular_values(sigma: np.ndarray, tol=1e-14, max_iter=50):
    """Solve min |d|^2 s.t. prod(sigma + d) = 1 by Newton's method on the KKT
    system  d + lam grad c(d) = 0, c(d) = 0  from d = 0, lam = 0.
    sigma: (..., 3).  Returns (s = sigma + d*, lam*) with shapes (..., 3), (...)."""
    sig = np.asarray(sigma, dtype=np.float64).reshape(-1, 3)
    N = sig.shape[0]
    d = np.zeros((N, 3))
    lam = np.zeros(N)
    active = np.ones(N, dtype=bool)
    for _ in range(max_iter):
        s = sig + d
        c = s[:, 0] * s[:, 1] * s[:, 2] - 1.0
        gc = np.stack([s[:, 1] * s[:, 2], s[:, 0] * s[:, 2], s[:, 0] * s[:, 1]], axis=1)
        r1 = d + lam[:, None] * gc
        active &= ~((np.abs(c) < tol) & (np.max(np.abs(r1), axis=1) < tol))
        if not np.any(active):
            break
        idx = np.flatnonzero(active)
        K = _kkt_matrix(s[idx], lam[idx], gc[idx])
        rhs = -np.concatenate([r1[idx], c[idx, None]], axis=1)
        step = np.linalg.solve(K, rhs[..., None])[..., 0]
        d[idx] += step[:, :3]
        lam[idx] += step[:, 3]
    return (sig + d).reshape(np.shape(sigma)), lam.reshape(np.shape(sigma)[:-1])


def _hess_c(s):
    z = np.zeros(s.shape[0])
    return np.stack([np.stack([z, s[:, 2], s[:, 1]], 1),
                     np.stack([s[:, 2], z, s[:, 0]], 1),
                     np.stack([s[:, 1], s[:, 0], z], 1)], 1)


def _kkt_matrix(s, lam, gc):
    K = np.zeros((s.shape[0], 4, 4))
    K[:, :3, :3] = np.eye(3)[None] + lam[:, None, None] * _hess_c(s)
    K[:, :3, 3] = gc
    K[:, 3, :3] = gc
    return K


def volume_ds_dsigma(s: np.ndarray, lam) -> np.ndarray:
    """ds/dsigma = I + dd*/dsigma from the differentiated KKT system (Eqn S5):
    [I + lam Hc, gc; gc^T, 0] [dd; dlam] = [-lam Hc dsigma; -gc^T dsigma].
    s: (..., 3), lam: (...).  Returns (..., 3, 3) with [i, j] = ds_i/dsigma_j."""
    sh = np.shape(s)
    s2 = np.asarray(s, dtype=np.float64).reshape(-1, 3)
    lam2 = np.asarray(lam, dtype=np.float64).reshape(-1)
    gc = np.stack([s2[:, 1] * s2[:, 2], s2[:, 0] * s2[:, 2], s2[:, 0] * s2[:, 1]], axis=1)
    hc = _hess_c(s2)
    K = _kkt_matrix(s2, lam2, gc)
    rhs = np.zeros((s2.shape[0], 4, 3))
    rhs[:, :3, :] = -lam2[:, None, None] * hc
    rhs[:, 3, :] = -gc
    sol = np.linalg.solve(K, rhs)
    return (np.eye(3)[None] + sol[:, :3, :]).reshape(sh + (3,))


def project_volume(F: np.ndarray) -> np.ndarray:
    """Batched volume-preserving projection D = U diag(s) V^T."""
    U, sig, V = signed_svd(F)
    s, _ = volume_singular_values(sig)
    return np.einsum("...ik,...k,...jk->...ij", U, s, V)


def isotropic_jacobian(U, sig, V, s, ds, eq_tol=1e-6):
    """Batched 9x9 Jacobians dP/dF (row-major vec) of P = U diag(s(sigma)) V^T.
    U, V: (N, 3, 3); sig, s: (N, 3); ds: (N, 3, 3).  Returns (N, 9, 9)."""
    N = U.shape[0]
    J = np.zeros((N, 9, 9))
    # divided differences a_ij and b_ij
    a = np.zeros((N, 3, 3))
    b = np.zeros((N, 3, 3))
    for i in range(3):
        for j in range(3):
            if i == j:
                continue
            dsig = sig[:, i] - sig[:, j]
            close = np.abs(dsig) <= eq_tol * np.maximum(1.0, np.abs(sig[:, i]))
            safe = np.where(close, 1.0, dsig)
            a[:, i, j] = np.where(close, ds[:, i, i] - ds[:, i, j], (s[:, i] - s[:, j]) / safe)
            b[:, i, j] = (s[:, i] + s[:, j]) / (sig[:, i] + sig[:, j])
    for col in range(9):
        r, c = col // 3, col % 3
        M = U[:, r, :, None] * V[:, c, None, :]            # M_kl = U[r,k] V[c,l]
        sym = 0.5 * (M + np.swapaxes(M, 1, 2))
        skw = 0.5 * (M - np.swapaxes(M, 1, 2))
        K = a * sym + b * skw
        diagM = np.diagonal(M, axis1=1, axis2=2)
        kd = np.einsum("nij,nj->ni", ds, diagM)
        K[:, [0, 1, 2], [0, 1, 2]] = kd
        J[:, :, col] = np.einsum("nik,nkl,njl->nij", U, K, V).reshape(N, 9)
    return J


def jacobian_corotated(F: np.ndarray) -> np.ndarray:
    """dR/dF as 9x9 matrices (row-major vec), F: (..., 3, 3) -> (..., 9, 9)."""
    sh = np.shape(F)[:-2]
    U, sig, V = signed_svd(np.asarray(F).reshape(-1, 3, 3))
    N = U.shape[0]
    J = isotropic_jacobian(U, sig, V, np.ones((N, 3)), np.zeros((N, 3, 3)))
    return J.reshape(sh + (9, 9))


def jacobian_volume(F: np.ndarray) -> np.ndarray:
    """dD/dF as 9x9 matrices (row-major vec), F: (..., 3, 3) -> (..., 9, 9)."""
    sh = np.shape(F)[:-2]
    U, sig, V = signed_svd(np.asarray(F).reshape(-1, 3, 3))
    s, lam = volume_singular_values(sig)
    J = isotropic_jacobian(U, sig, V, s, volume_ds_dsigma(s, lam))
    return J.reshape(sh + (9, 9))


def project_muscle(f: np.ndarray, a) -> np.ndarray:
    """p = (1 - a) f / |f|, batched over leading axes of f (..., 3)."""
    nrm = np.linalg.norm(f, axis=-1, keepdims=True)
    return (1.0 - np.asarray(a))[..., None] * f / nrm


def jacobian_muscle(f: np.ndarray, a: float) -> np.ndarray:
    """dp/df = (1 - a)/|f| (I - fhat fhat^T)."""
    nrm = np.linalg.norm(f)
    fh = f / nrm
    return (1.0 - a) / nrm * (np.eye(3) - np.outer(fh, fh))


def project_ground(x: np.ndarray) -> np.ndarray:
    """Penalty contact with the ground half-space z >= 0."""
    p = np.array(x, dtype=np.float64, copy=True)
    p[..., 2] = np.maximum(p[..., 2], 0.0)
    return p
