"""Voxel meshes and their FEM operators (oracle; test infrastructure only).

Sec. 3 ("Projective Dynamics") takes G_c as the discrete operator mapping
nodal positions x to the deformation gradient F of a finite element; the
supplement ("Background elasticity") evaluates the energy density at the
element's Gaussian quadrature points.  Two element rules on the kept cells of a
voxel grid:
  * "hex8": trilinear hexahedra, 2x2x2 Gauss points xi_q in
    {-1/sqrt3, +1/sqrt3}^3, each with volume weight V_q = dx^3 / 8; lumped mass
    m_j = sum over cells touching j of rho dx^3 / 8 (Sec. 3, "M a lumped mass
    matrix");
  * "tet6": every cell split into six linear tetrahedra around its diagonal from
    corner (0,0,0) to corner (1,1,1) (one per order of the three axes; the split
    is conforming between neighbouring cells), one point per tetrahedron with
    weight V = dx^3 / 6 (a linear element has a constant F); lumped mass rho V / 4
    per vertex of each tetrahedron.  The paper simulates tetrahedral meshes
    (Secs. 5.1, 7) whose assets are not available; this rule is the voxel stand-in.
Readings (the paper is silent): the quadrature of each rule, the lumping.
Both rules express each point's shape-function gradients over all 8 corners of
its cell (zero for corners outside a tetrahedron), so G_c x_e has one form.
"""
from __future__ import annotations

import numpy as np


class VoxelMesh:
    """Regular voxel mesh: kept cells of an nx*ny*nz grid with edge dx.

    Attributes
      X      (n, 3) rest positions of kept nodes (increasing grid id)
      elems  (e, 8) kept-node indices of each kept cell's corners
      grid   (n,)   grid id of each kept node
      gradN  (Q, 8, 3) d N_a / d X at point q: gradN[q, a, :] (Q = 8 or 6)
      Vq     volume weight of every point: dx^3 / 8 (hex8) or dx^3 / 6 (tet6)
    """

    def __init__(self, nx, ny, nz, dx, origin=(0.0, 0.0, 0.0), cell_mask=None, rule="hex8"):
        assert rule in ("hex8", "tet6")
        self.rule = rule
        self.nx, self.ny, self.nz, self.dx = int(nx), int(ny), int(nz), float(dx)
        cells = []
        for ci in range(nx):
            for cj in range(ny):
                for ck in range(nz):
                    cid = (ci * ny + cj) * nz + ck
                    if cell_mask is not None and not cell_mask[cid]:
                        continue
                    corners = []
                    for a in range(8):
                        di, dj, dk = (a >> 2) & 1, (a >> 1) & 1, a & 1
                        corners.append(((ci + di) * (ny + 1) + (cj + dj)) * (nz + 1) + (ck + dk))
                    cells.append(corners)
        cells = np.array(cells, dtype=np.int64).reshape(-1, 8)
        self.grid = np.unique(cells.ravel())
        lookup = {g: i for i, g in enumerate(self.grid.tolist())}
        self.elems = np.vectorize(lookup.__getitem__)(cells).astype(np.int64).reshape(-1, 8)
        k = self.grid % (nz + 1)
        j = (self.grid // (nz + 1)) % (ny + 1)
        i = self.grid // ((nz + 1) * (ny + 1))
        self.ijk = np.stack([i, j, k], axis=1)
        self.X = self.ijk.astype(np.float64) * dx + np.asarray(origin, dtype=np.float64)
        if rule == "hex8":
            self.gradN = shape_gradients(dx)
            self.Vq = dx ** 3 / 8.0
        else:
            self.gradN, vols = tet_shape_gradients(dx)
            self.Vq = float(vols[0])

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def e(self) -> int:
        return self.elems.shape[0]

    def lumped_mass(self, rho: float) -> np.ndarray:
        m = np.zeros(self.n)
        if self.rule == "hex8":
            np.add.at(m, self.elems.ravel(), rho * self.dx ** 3 / 8.0)
        else:
            for tet in kuhn_tetrahedra():
                for a in tet:
                    np.add.at(m, self.elems[:, a], rho * self.Vq / 4.0)
        return m

    def deformation_gradients(self, x: np.ndarray) -> np.ndarray:
        """F[e, q] = sum_a x_a (outer) gradN[q, a]   ->  shape (e, 8, 3, 3)."""
        xe = x[self.elems]                       # (e, 8 corners, 3)
        return np.einsum("eai,qaj->eqij", xe, self.gradN)

    def G_matrix(self) -> np.ndarray:
        """The 9x24 operator G_q of every point, (Q, 9, 24): vec(F) =
        G_q x_e with vec row-major (i*3+j) and x_e node-major (a*3+i)."""
        Q = self.gradN.shape[0]
        G = np.zeros((Q, 9, 24))
        for q in range(Q):
            for a in range(8):
                for i in range(3):
                    for j in range(3):
                        G[q, i * 3 + j, a * 3 + i] = self.gradN[q, a, j]
        return G


def shape_gradients(dx: float) -> np.ndarray:
    """Gradients of the trilinear shape functions N_a(xi) = prod_d (1 + s_ad xi_d)/2
    on the reference cube [-1, 1]^3, mapped to a cube of edge dx (dxi/dX = 2/dx)."""
    g = 1.0 / np.sqrt(3.0)
    out = np.zeros((8, 8, 3))
    for q in range(8):
        xi = np.array([(2 * ((q >> 2) & 1) - 1) * g, (2 * ((q >> 1) & 1) - 1) * g,
                       (2 * (q & 1) - 1) * g])
        for a in range(8):
            s = np.array([2 * ((a >> 2) & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * (a & 1) - 1],
                         dtype=np.float64)
            f = (1.0 + s * xi) / 2.0
            for d in range(3):
                prod = 1.0
                for d2 in range(3):
                    if d2 != d:
                        prod *= f[d2]
                out[q, a, d] = (s[d] / 2.0) * prod * (2.0 / dx)
    return out


def kuhn_tetrahedra():
    """The six tetrahedra of a cell as corner indices (a = 4 di + 2 dj + dk):
    for each order (p1, p2, p3) of the axes, the path from corner 0 along p1,
    then p2, then p3 to corner 7."""
    out = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        c1 = 4 >> perm[0]
        c2 = c1 + (4 >> perm[1])
        out.append((0, c1, c2, 7))
    return out


def tet_shape_gradients(dx: float):
    """Gradients of the barycentric coordinates of each Kuhn tetrahedron over the
    8 corners of a cube of edge dx, (6, 8, 3), and the six volumes: with E the
    edge matrix [P1 - P0, P2 - P0, P3 - P0], the coordinates l_1..3 = E^-1 (X - P0)
    and l_0 = 1 - l_1 - l_2 - l_3."""
    corner = np.array([[(a >> 2) & 1, (a >> 1) & 1, a & 1] for a in range(8)], dtype=np.float64) * dx
    grads = np.zeros((6, 8, 3))
    vols = np.zeros(6)
    for t, tet in enumerate(kuhn_tetrahedra()):
        P = corner[list(tet)]
        E = (P[1:] - P[0]).T
        B = np.linalg.inv(E)
        for i in range(3):
            grads[t, tet[i + 1]] = B[i]
        grads[t, tet[0]] = -B.sum(axis=0)
        vols[t] = abs(np.linalg.det(E)) / 6.0
    return grads, vols
