"""Unstructured tetrahedral meshes (oracle; test infrastructure only).

Secs. 5.1 and 7 simulate tetrahedral meshes (the duck, the tennis balls) built from
surface meshes that are not available here; the voxel split of oracle/mesh.py
(rule "tet6") keeps the grid's nodes, and this module covers meshes with their own
node sets.  Each element is a linear tetrahedron (X_0, X_1, X_2, X_3): with the edge
matrix D = [X_1 - X_0, X_2 - X_0, X_3 - X_0] the barycentric coordinates are
l_{1..3} = D^-1 (X - X_0), l_0 = 1 - l_1 - l_2 - l_3, so grad N_a is row a - 1 of
D^-1 for a = 1..3 and grad N_0 = -(their sum); F = sum_a x_a (outer) grad N_a is
constant on the element, one point of weight V = det(D) / 6 (> 0: vertices ordered
so), lumped mass rho V / 4 per vertex (reading, as for the voxel split).

TetModel is the PD model of oracle/model.py (corotated and volume energies, the PD
matrix A, gravity, external force, penalty ground contact with friction on the
scene's candidate nodes; no muscles) on such a mesh; it
keeps Model's interface so that newton.py, pd_cpu.py and adjoint.py run on it.
With `scene.neohookean` the corotated and volume terms give way to the Neo-Hookean
energy of oracle/neohookean.py (Sec. 8; the paper's Armadillo is such a mesh) with
mu = w_corot/2, lambda = w_vol, as in oracle/model.py.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import neohookean as nh
from . import projections as pj
from .model import Model, lame_weights


class TetMesh:
    """Attributes: X (n, 3) rest positions, elems (e, 4) vertex indices (positively
    oriented), gradN (e, 1, 4, 3), Vq (e,) element volumes."""

    def __init__(self, X, tets):
        self.X = np.asarray(X, dtype=np.float64)
        T = np.asarray(tets, dtype=np.int64).reshape(-1, 4).copy()
        D = np.stack([self.X[T[:, a]] - self.X[T[:, 0]] for a in (1, 2, 3)], axis=2)   # columns
        det = np.linalg.det(D)
        flip = det < 0
        T[flip, 1], T[flip, 2] = T[flip, 2].copy(), T[flip, 1].copy()
        D = np.stack([self.X[T[:, a]] - self.X[T[:, 0]] for a in (1, 2, 3)], axis=2)
        self.elems = T
        self.Vq = np.linalg.det(D) / 6.0
        assert np.all(self.Vq > 0), "degenerate tetrahedron"
        B = np.linalg.inv(D)                              # row i = grad l_{i+1}
        g = np.zeros((T.shape[0], 1, 4, 3))
        g[:, 0, 1:, :] = B
        g[:, 0, 0, :] = -B.sum(axis=1)
        self.gradN = g

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def e(self) -> int:
        return self.elems.shape[0]

    @property
    def dx(self) -> float:
        """A length scale for tolerances that voxel meshes take from their cell edge:
        the edge of a cube of six times the mean tetrahedron volume."""
        return float(np.cbrt(6.0 * self.Vq.mean()))

    def lumped_mass(self, rho: float) -> np.ndarray:
        m = np.zeros(self.n)
        for a in range(4):
            np.add.at(m, self.elems[:, a], rho * self.Vq / 4.0)
        return m

    def deformation_gradients(self, x: np.ndarray) -> np.ndarray:
        """F[e, 0] = sum_a x_a (outer) grad N_a, shape (e, 1, 3, 3)."""
        return np.einsum("eai,eqaj->eqij", x[self.elems], self.gradN)

    def G_matrices(self) -> np.ndarray:
        """(e, 1, 9, 12): vec(F) = G x_e, vec row-major (3 i + j), x_e node-major (3 a + i)."""
        G = np.zeros((self.e, 1, 9, 12))
        for a in range(4):
            for i in range(3):
                for j in range(3):
                    G[:, 0, 3 * i + j, 3 * a + i] = self.gradN[:, 0, a, j]
        return G


class TetModel(Model):
    """The PD model on an unstructured tetrahedral mesh (scene: workloads.TetScene)."""

    def __init__(self, scene, youngs=None, poisson=None, mu=None):
        s = scene
        self.scene = s
        self.mesh = TetMesh(s.X, s.tets)
        mesh = self.mesh
        assert mesh.n == s.x0.shape[0]
        E = np.asarray(s.youngs if youngs is None else youngs, dtype=np.float64)
        self.youngs = E
        self.poisson = float(s.poisson if poisson is None else poisson)
        wc, wv = lame_weights(E, self.poisson)
        self.w_corot = wc if s.corotated else np.zeros(mesh.e)
        self.w_vol = wv if s.volume else np.zeros(mesh.e)
        self.w_musc = np.zeros(mesh.e)
        self.fiber = np.zeros((mesh.e, 3))
        self.m = mesh.lumped_mass(s.density)
        self.h = float(s.h)
        self.gravity = np.asarray(s.gravity, dtype=np.float64)
        self.k = float(getattr(s, "k_contact", 0.0))
        self.mu = float(getattr(s, "mu", 0.0) if mu is None else mu)
        c = getattr(s, "contact", None)
        self.contact = np.zeros(mesh.n, dtype=bool) if c is None else np.asarray(c, dtype=bool)
        self.dirichlet = np.asarray(s.dirichlet, dtype=bool)
        self.free_nodes = np.flatnonzero(~self.dirichlet)
        self.free_dofs = (self.free_nodes[:, None] * 3 + np.arange(3)[None, :]).ravel()
        self.G = mesh.G_matrices()
        self.neohookean = bool(getattr(s, "neohookean", False))
        if self.neohookean:
            self.nh_mu = 0.5 * wc
            self.nh_lam = wv

    def energy(self, x, act=None, loc=None):
        loc = self.local(x, act) if loc is None else loc
        F = loc["F"]
        V = self.mesh.Vq[:, None]
        E = 0.0
        if "psi_nh" in loc:
            E += np.sum(V * loc["psi_nh"])
        if "R" in loc:
            E += 0.5 * np.sum(self.w_corot[:, None] * V * np.sum((F - loc["R"]) ** 2, axis=(2, 3)))
        if "D" in loc:
            E += 0.5 * np.sum(self.w_vol[:, None] * V * np.sum((F - loc["D"]) ** 2, axis=(2, 3)))
        if self.k > 0:   # k/2 |x_j - p(x_j)|^2, p = (x, y, max(z, 0)) on the candidates
            E += 0.5 * self.k * np.sum(np.minimum(x[self.contact, 2], 0.0) ** 2)
        return E

    def grad_E(self, x, act=None, loc=None):
        loc = self.local(x, act) if loc is None else loc
        F = loc["F"]
        S = np.zeros_like(F)
        if "P_nh" in loc:
            S += self.mesh.Vq[:, None, None, None] * loc["P_nh"]
        if "R" in loc:
            S += (self.w_corot * self.mesh.Vq)[:, None, None, None] * (F - loc["R"])
        if "D" in loc:
            S += (self.w_vol * self.mesh.Vq)[:, None, None, None] * (F - loc["D"])
        fe = np.einsum("eqij,eqaj->eai", S, self.mesh.gradN)    # (e, 4, 3)
        g = np.zeros_like(x)
        np.add.at(g, self.mesh.elems.ravel(), fe.reshape(-1, 3))
        if self.k > 0:
            g[:, 2] += np.where(self.contact, self.k * np.minimum(x[:, 2], 0.0), 0.0)
        return g

    def _element_blocks(self, x, act=None, linearised=True):
        """Per-element 12x12: V w G^T (I - J) G (or V w G^T G when linearised=False);
        Neo-Hookean: V G^T T G with the tangent T = dP/dF."""
        G = self.G                                         # (e, 1, 9, 12)
        V = self.mesh.Vq
        if self.neohookean and linearised:
            F = self.mesh.deformation_gradients(x)
            mu = np.broadcast_to(self.nh_mu[:, None], F.shape[:2])
            lam = np.broadcast_to(self.nh_lam[:, None], F.shape[:2])
            return np.einsum("e,eqki,eqkl,eqlj->eij", V, G, nh.tangent(F, mu, lam), G)
        blocks = np.einsum("e,eqki,eqkj->eij", (self.w_corot + self.w_vol) * V, G, G)
        if not linearised:
            return blocks
        F = self.local(x, act)["F"]
        J = np.zeros((self.mesh.e, 1, 9, 9))
        if np.any(self.w_corot):
            J += self.w_corot[:, None, None, None] * pj.jacobian_corotated(F)
        if np.any(self.w_vol):
            J += self.w_vol[:, None, None, None] * pj.jacobian_volume(F)
        return blocks - np.einsum("e,eqki,eqkl,eqlj->eij", V, G, J, G)

    def _assemble(self, blocks, contact_diag):
        mesh = self.mesh
        n3 = 3 * mesh.n
        dofs = (mesh.elems[:, :, None] * 3 + np.arange(3)[None, None, :]).reshape(mesh.e, 12)
        rows = np.repeat(dofs, 12, axis=1).ravel()
        cols = np.tile(dofs, (1, 12)).ravel()
        K = sp.coo_matrix((blocks.ravel(), (rows, cols)), shape=(n3, n3)).tocsr()
        diag = np.repeat(self.m / self.h ** 2, 3) + contact_diag
        return (K + sp.diags(diag)).tocsr()
