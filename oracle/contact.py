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
