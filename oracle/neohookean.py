"""Compressible Neo-Hookean material (oracle; test infrastructure only).

Sec. 8 of the paper runs DiffPD with the Neo-Hookean model (the twisting
armadillo) without printing its energy; reading: the standard compressible form
per unit rest volume

  psi(F) = mu/2 (tr(F^T F) - 3) - mu log J + lambda/2 (log J)^2,   J = det F,

with mu = w_corot / 2 and lambda = w_vol (the Lame parameters of the element's
(E, nu)), whose first Piola-Kirchhoff stress is

  P(F) = d psi / dF = mu (F - F^-T) + lambda log J F^-T

and whose Hessian applied to dF is

  dP = mu dF + (mu - lambda log J) F^-T dF^T F^-T + lambda tr(F^-1 dF) F^-T.

Plain NumPy on (..., 3, 3) arrays, FP64.
"""
from __future__ import annotations

import numpy as np


def energy_density(F, mu, lam):
    """psi(F) per unit rest volume; mu, lam broadcast against F[..., 0, 0]."""
    J = np.linalg.det(F)
    logJ = np.log(J)
    I1 = np.einsum("...ij,...ij->...", F, F)
    return 0.5 * mu * (I1 - 3.0) - mu * logJ + 0.5 * lam * logJ ** 2


def first_piola(F, mu, lam):
    """P(F) = mu (F - F^-T) + lam log J F^-T."""
    FinvT = np.swapaxes(np.linalg.inv(F), -1, -2)
    logJ = np.log(np.linalg.det(F))
    mu = np.asarray(mu)[..., None, None]
    lam = np.asarray(lam)[..., None, None]
    return mu * (F - FinvT) + lam * logJ[..., None, None] * FinvT


def dpiola(F, dF, mu, lam):
    """dP(F)[dF] = mu dF + (mu - lam log J) F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T."""
    Finv = np.linalg.inv(F)
    FinvT = np.swapaxes(Finv, -1, -2)
    logJ = np.log(np.linalg.det(F))
    mu = np.asarray(mu)[..., None, None]
    lam = np.asarray(lam)[..., None, None]
    tr = np.einsum("...ij,...ji->...", Finv, dF)
    return (mu * dF + (mu - lam * logJ[..., None, None]) * (FinvT @ np.swapaxes(dF, -1, -2) @ FinvT)
            + lam * tr[..., None, None] * FinvT)


def tangent(F, mu, lam):
    """(..., 9, 9) matrix T with vec(dP) = T vec(dF), vec row-major (index 3 i + j)."""
    T = np.zeros(F.shape[:-2] + (9, 9))
    for k in range(9):
        E = np.zeros(F.shape)
        E[..., k // 3, k % 3] = 1.0
        T[..., :, k] = dpiola(F, E, mu, lam).reshape(F.shape[:-2] + (9,))
    return T
