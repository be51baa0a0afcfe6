"""The discrete PD model: energy, gradient, Hessian and the PD matrix A
(oracle; test infrastructure only).

  g(x)      = (x - y)^T M (x - y) / (2 h^2) + E(x)                    (Eqn 5)
  E(x)      = sum_c w_c/2 |G_c x - p_c(x)|^2, p_c = Proj_{M_c}(G_c x)   (Eqns 16-17)
  grad E    = sum_c w_c G_c^T (G_c x - p_c)                            (Eqn 20)
  Hess E    = sum_c w_c G_c^T (I - dp_c/dx) G_c                        (Eqn 21)
  A         = M/h^2 + sum_c w_c G_c^T G_c                              (Eqn 19)

Energy set per quadrature point q of element e (weights per unit volume times
V_q = dx^3/8 for hexahedra, dx^3/6 per tetrahedron of the tet6 rule): corotated w = E/(1+nu) (= 2 mu), volume-preserving
w = E nu/((1+nu)(1-2nu)) (= lambda), muscle w = E on fibre elements; penalty
contact w = k per candidate node.  (Reading: the paper does not state the
map from (E, nu) to w.)
Neo-Hookean scenes (Sec. 8, `scene.neohookean`): the corotated and volume terms of
E are replaced by the Neo-Hookean energy (oracle/neohookean.py) with mu = w_corot/2,
lambda = w_vol; E is then not a PD energy, its Hessian is assembled from the
Neo-Hookean tangent, and A keeps the PD matrix of the same weights.
Penalty friction (Sec. 5.1) enters f_ext: reading, per candidate node j with
z_j < 0 at the start of the step, f_n = k (-z_j), v_t = (v_x, v_y),
f_t = -min(mu f_n, m_j |v_t| / h) v_t / |v_t| (zero when |v_t| = 0).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import VoxelMesh
from . import neohookean as nh
from . import projections as pj


def lame_weights(E, nu):
    """(w_corotated, w_volume) per unit volume from Young's modulus and Poisson's ratio."""
    E = np.asarray(E, dtype=np.float64)
    return E / (1.0 + nu), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


class Model:
    def __init__(self, scene, youngs=None, poisson=None, mu=None):
        s = scene
        self.scene = s
        self.mesh = VoxelMesh(s.nx, s.ny, s.nz, s.dx, s.origin, s.cell_mask,
                              rule=getattr(s, "element_rule", "hex8"))
        mesh = self.mesh
        assert mesh.n == s.x0.shape[0]
        E = np.asarray(s.youngs if youngs is None else youngs, dtype=np.float64)
        self.youngs = E
        self.poisson = float(s.poisson if poisson is None else poisson)
        wc, wv = lame_weights(E, self.poisson)
        self.w_corot = wc if s.corotated else np.zeros(mesh.e)
        self.w_vol = wv if s.volume else np.zeros(mesh.e)
        if s.muscle is not None:
            self.w_musc = E * np.asarray(s.muscle, dtype=np.float64)
            self.fiber = np.asarray(s.fiber, dtype=np.float64)
        else:
            self.w_musc = np.zeros(mesh.e)
            self.fiber = np.zeros((mesh.e, 3))
        self.m = mesh.lumped_mass(s.density)
        self.h = float(s.h)
        self.gravity = np.asarray(s.gravity, dtype=np.float64)
        self.k = float(s.k_contact)
        self.mu = float(s.mu if mu is None else mu)
        self.contact = np.asarray(s.contact, dtype=bool)
        self.dirichlet = np.asarray(s.dirichlet, dtype=bool)
        self.free_nodes = np.flatnonzero(~self.dirichlet)
        self.free_dofs = (self.free_nodes[:, None] * 3 + np.arange(3)[None, :]).ravel()
        self.G = mesh.G_matrix()
        self.neohookean = bool(getattr(s, "neohookean", False))
        if self.neohookean:
            self.nh_mu = 0.5 * wc
            self.nh_lam = wv

    # ---------------------------------------------------------------- local
    def local(self, x, act=None):
        """Deformation gradients and projections at every Gauss point."""
        F = self.mesh.deformation_gradients(x)                 # (e, 8, 3, 3)
        out = {"F": F}
        if self.neohookean:
            mu = np.broadcast_to(self.nh_mu[:, None], F.shape[:2])
            lam = np.broadcast_to(self.nh_lam[:, None], F.shape[:2])
            out["P_nh"] = nh.first_piola(F, mu, lam)
            out["psi_nh"] = nh.energy_density(F, mu, lam)
        else:
            if np.any(self.w_corot):
                out["R"] = pj.project_corotated(F)
            if np.any(self.w_vol):
                out["D"] = pj.project_volume(F)
        if np.any(self.w_musc):
            f = np.einsum("eqij,ej->eqi", F, self.fiber)
            a = np.zeros(self.mesh.e) if act is None else np.asarray(act, dtype=np.float64)
            out["f"] = f
            out["pm"] = pj.project_muscle(f, np.broadcast_to(a[:, None], f.shape[:2]))
            out["a"] = a
        return out

    def energy(self, x, act=None, loc=None):
        loc = self.local(x, act) if loc is None else loc
        F = loc["F"]
        Vq = self.mesh.Vq
        E = 0.0
        if "psi_nh" in loc:
            E += Vq * np.sum(loc["psi_nh"])
        if "R" in loc:
            E += 0.5 * Vq * np.sum(self.w_corot[:, None] * np.sum((F - loc["R"]) ** 2, axis=(2, 3)))
        if "D" in loc:
            E += 0.5 * Vq * np.sum(self.w_vol[:, None] * np.sum((F - loc["D"]) ** 2, axis=(2, 3)))
        if "f" in loc:
            E += 0.5 * Vq * np.sum(self.w_musc[:, None] * np.sum((loc["f"] - loc["pm"]) ** 2, axis=2))
        if self.k > 0:
            z = x[self.contact, 2]
            E += 0.5 * self.k * np.sum(np.minimum(z, 0.0) ** 2)
        return E

    def grad_E(self, x, act=None, loc=None):
        """grad E = sum_c w_c G_c^T (G_c x - p_c), shape (n, 3)."""
        loc = self.local(x, act) if loc is None else loc
        F = loc["F"]
        Vq = self.mesh.Vq
        S = np.zeros_like(F)                                   # stress-like (e,q,3,3)
        if "P_nh" in loc:
            S += Vq * loc["P_nh"]
        if "R" in loc:
            S += (self.w_corot * Vq)[:, None, None, None] * (F - loc["R"])
        if "D" in loc:
            S += (self.w_vol * Vq)[:, None, None, None] * (F - loc["D"])
        if "f" in loc:
            r = (self.w_musc * Vq)[:, None, None] * (loc["f"] - loc["pm"])   # (e,q,3)
            S += np.einsum("eqi,ej->eqij", r, self.fiber)
        fe = np.einsum("eqij,qaj->eai", S, self.mesh.gradN)    # (e, 8, 3)
        g = np.zeros_like(x)
        np.add.at(g, self.mesh.elems.ravel(), fe.reshape(-1, 3))
        if self.k > 0:
            z = x[:, 2]
            g[:, 2] += np.where(self.contact, self.k * np.minimum(z, 0.0), 0.0)
        return g

    # --------------------------------------------------------------- global
    def _element_blocks(self, x, act=None, linearised=True):
        """Per-element 24x24 matrices sum_q w V_q G_q^T (I - J_q) G_q (or
        sum_q w V_q G_q^T G_q when linearised=False, which gives A)."""
        mesh = self.mesh
        G = self.G
        Vq = mesh.Vq
        GtG = np.einsum("qki,qkj->qij", G, G)                  # (8, 24, 24)
        if self.neohookean and linearised:
            # Hess E of the Neo-Hookean terms: sum_q V_q G_q^T T_q G_q
            F = mesh.deformation_gradients(x)
            mu = np.broadcast_to(self.nh_mu[:, None], F.shape[:2])
            lam = np.broadcast_to(self.nh_lam[:, None], F.shape[:2])
            blocks = Vq * np.einsum("qki,eqkl,qlj->eij", G, nh.tangent(F, mu, lam), G)
        else:
            blocks = np.einsum("e,qij->eij", (self.w_corot + self.w_vol) * Vq, GtG)
        if np.any(self.w_musc):
            Q = G.shape[0]
            Gm = np.zeros((mesh.e, Q, 3, 24))
            for q in range(Q):
                Gq = G[q].reshape(3, 3, 24)                    # [i, j, dof]
                Gm[:, q] = np.einsum("ijd,ej->eid", Gq, self.fiber)
            blocks = blocks + np.einsum("e,eqki,eqkj->eij", self.w_musc * Vq, Gm, Gm)
        if not linearised:
            return blocks
        loc = self.local(x, act)
        F = loc["F"]
        if not self.neohookean:
            J = np.zeros((mesh.e, G.shape[0], 9, 9))
            if np.any(self.w_corot):
                J += self.w_corot[:, None, None, None] * pj.jacobian_corotated(F)
            if np.any(self.w_vol):
                J += self.w_vol[:, None, None, None] * pj.jacobian_volume(F)
            blocks = blocks - Vq * np.einsum("qki,eqkl,qlj->eij", G, J, G)
        if np.any(self.w_musc):
            f = loc["f"]
            nrm = np.linalg.norm(f, axis=2)
            fh = f / nrm[..., None]
            Jm = ((1.0 - loc["a"])[:, None, None, None] / nrm[..., None, None]
                  * (np.eye(3)[None, None] - fh[..., :, None] * fh[..., None, :]))
            blocks = blocks - np.einsum("e,eqki,eqkl,eqlj->eij", self.w_musc * Vq, Gm, Jm, Gm)
        return blocks

    def _assemble(self, blocks, contact_diag):
        mesh = self.mesh
        n3 = 3 * mesh.n
        dofs = (mesh.elems[:, :, None] * 3 + np.arange(3)[None, None, :]).reshape(mesh.e, 24)
        rows = np.repeat(dofs, 24, axis=1).ravel()
        cols = np.tile(dofs, (1, 24)).ravel()
        K = sp.coo_matrix((blocks.ravel(), (rows, cols)), shape=(n3, n3)).tocsr()
        diag = np.repeat(self.m / self.h ** 2, 3) + contact_diag
        return (K + sp.diags(diag)).tocsr()

    def hessian(self, x, act=None):
        """Hess g = M/h^2 + Hess E (Eqns 13, 21), full 3n x 3n sparse."""
        cd = np.zeros(3 * self.mesh.n)
        if self.k > 0:
            pen = self.contact & (x[:, 2] < 0.0)
            cd[np.flatnonzero(pen) * 3 + 2] = self.k
        return self._assemble(self._element_blocks(x, act, True), cd)

    def A_matrix(self):
        """A = M/h^2 + sum_c w_c G_c^T G_c (Eqn 19), full 3n x 3n sparse."""
        cd = np.zeros(3 * self.mesh.n)
        if self.k > 0:
            cd[(np.flatnonzero(self.contact)[:, None] * 3 + np.arange(3)).ravel()] = self.k
        return self._assemble(self._element_blocks(None, None, False), cd)

    # ------------------------------------------------------------- friction
    def friction(self, x, v, mu=None):
        """Penalty friction force (added to f_ext), from the state at the start of the step."""
        mu = self.mu if mu is None else mu
        f = np.zeros_like(x)
        if self.k <= 0:
            return f
        for j in np.flatnonzero(self.contact):
            z = x[j, 2]
            if z >= 0.0:
                continue
            fn = self.k * (-z)
            vt = v[j, :2]
            nv = np.linalg.norm(vt)
            if nv == 0.0:
                continue
            mag = min(mu * fn, self.m[j] * nv / self.h)
            f[j, :2] = -mag * vt / nv
        return f

    def friction_vjp(self, x, v, gf, mu=None):
        """Given dL/df_fric (n,3), return (dL/dx, dL/dv, dL/dmu) through the friction force."""
        mu = self.mu if mu is None else mu
        gx = np.zeros_like(x)
        gv = np.zeros_like(v)
        gmu = 0.0
        if self.k <= 0:
            return gx, gv, gmu
        for j in np.flatnonzero(self.contact):
            z = x[j, 2]
            if z >= 0.0:
                continue
            fn = self.k * (-z)
            vt = v[j, :2]
            nv = np.linalg.norm(vt)
            if nv == 0.0:
                continue
            t = vt / nv
            gt = gf[j, :2]
            if mu * fn < self.m[j] * nv / self.h:
                # f_t = -mu k (-z) t = mu k z t
                gx[j, 2] += mu * self.k * (gt @ t)
                gmu += self.k * z * (gt @ t)
                gv[j, :2] += mu * self.k * z * (np.eye(2) - np.outer(t, t)) @ gt / nv
            else:
                # f_t = -m v_t / h
                gv[j, :2] += -self.m[j] / self.h * gt
        return gx, gv, gmu

    # ------------------------------------------------------------ helpers
    def predictor(self, x, v, f_ext, mu=None):
        f = f_ext + self.m[:, None] * self.gravity[None, :] + self.friction(x, v, mu)
        return x + self.h * v + self.h ** 2 * f / self.m[:, None]

    def g_value(self, x, y, act=None, loc=None):
        d = (x - y)[self.free_nodes]
        return 0.5 / self.h ** 2 * np.sum(self.m[self.free_nodes, None] * d * d) + self.energy(x, act, loc)

    def grad_g(self, x, y, act=None, loc=None):
        """grad g = M (x - y)/h^2 + grad E restricted to free DoFs, (n_free*3,)."""
        g = self.m[:, None] * (x - y) / self.h ** 2 + self.grad_E(x, act, loc)
        return g[self.free_nodes].ravel()
