"""Seeded unstructured tetrahedral scenes (input generators only).

The paper's tetrahedral meshes (Secs. 5.1, 7) come from surface meshes that are not
available; these stand-ins have their own node sets: a box of jittered lattice
points (the faces' points stay on their faces, so the hull is the box) split into
tetrahedra by a Delaunay triangulation.  Streams: PCG64 with seed = index * 1000 +
stream, as in scenes.py.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
from scipy.spatial import Delaunay


@dataclasses.dataclass
class TetScene:
    name: str
    X: np.ndarray                     # (n, 3) rest positions
    tets: np.ndarray                  # (e, 4) vertex indices
    density: float
    youngs: np.ndarray                # (e,) Young's modulus per tetrahedron [Pa]
    poisson: float
    corotated: bool
    volume: bool
    dirichlet: np.ndarray             # (n,) uint8: fixed at the rest position
    gravity: np.ndarray               # (3,)
    h: float
    T: int
    x0: np.ndarray                    # (n, 3)
    v0: np.ndarray                    # (n, 3)
    f_ext: np.ndarray                 # (n, 3)
    loss_w: np.ndarray                # (n, 3)
    tol_fwd: float
    tol_bwd: float
    act: Optional[np.ndarray] = None
    muscle: Optional[np.ndarray] = None   # no muscle fibres on these meshes
    contact: Optional[np.ndarray] = None  # (n,) uint8: penalty-contact candidate, None = none
    neohookean: bool = False              # Neo-Hookean material in place of corotated + volume
    k_contact: float = 0.0
    mu: float = 0.0


def _rng(index: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(index * 1000 + stream))


def unstructured_tet_beam(nx=6, ny=3, nz=3, *, T=4, index=11, dx=0.01, jitter=0.3, E=1e5,
                          nu=0.45, volume=True) -> TetScene:
    """Cantilever of (nx+1)(ny+1)(nz+1) lattice points of spacing dx, each moved by
    U(-jitter, jitter) dx along the axes it is not held on by a face of the box,
    Delaunay-tetrahedralised (tetrahedra of volume < 1e-6 dx^3 on the hull dropped);
    the x = 0 face fixed, gravity, stiffness E exp(0.2 N(0,1)) per tetrahedron,
    v0 ~ N(0, 0.01^2), loss weights N(0, 1)."""
    g = np.stack(np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij"),
                 axis=-1).reshape(-1, 3).astype(np.float64)
    dims = np.array([nx, ny, nz], dtype=np.float64)
    movable = (g > 0) & (g < dims[None, :])
    X = (g + jitter * _rng(index, 1).uniform(-1.0, 1.0, g.shape) * movable) * dx
    tri = Delaunay(X)
    tets = tri.simplices.astype(np.int64)
    D = np.stack([X[tets[:, a]] - X[tets[:, 0]] for a in (1, 2, 3)], axis=2)
    vol = np.abs(np.linalg.det(D)) / 6.0
    tets = tets[vol > 1e-6 * dx ** 3]
    n, e = X.shape[0], tets.shape[0]
    dirichlet = (g[:, 0] == 0).astype(np.uint8)
    v0 = 0.01 * _rng(index, 2).standard_normal((n, 3))
    v0[dirichlet.astype(bool)] = 0.0
    return TetScene(name=f"unstructured_tet_beam_{nx}x{ny}x{nz}", X=X, tets=tets, density=1e3,
                    youngs=E * np.exp(0.2 * _rng(index, 3).standard_normal(e)), poisson=nu,
                    corotated=True, volume=volume, dirichlet=dirichlet,
                    gravity=np.array([0.0, 0.0, -9.81]), h=0.01, T=T, x0=X.copy(), v0=v0,
                    f_ext=np.zeros((n, 3)), loss_w=_rng(index, 4).standard_normal((n, 3)),
                    tol_fwd=1e-10, tol_bwd=1e-10)


def unstructured_tet_ball(T: int = 20, *, index: int = 12, R: float = 3.2, dx: float = 0.01,
                          jitter: float = 0.25, E: float = 1e5) -> TetScene:
    """Ball of the lattice points (i, j, k) dx with |(i, j, k)| <= R, each moved by
    U(-jitter, jitter) dx per axis, Delaunay-tetrahedralised (tetrahedra of volume
    < 1e-6 dx^3 dropped, with the nodes left in none): stands in for the tennis
    balls of Sec. 7 (a 320-tetrahedron sphere mesh); its lowest node 2 mm above the
    ground z = 0, moving at (0.2, 0, -0.3) m/s plus N(0, 0.01^2) per DoF, penalty
    contact k = 1e4 N/m on the convex-hull nodes with Coulomb friction mu = 0.4,
    E = 1e5, nu = 0.45, h = 0.005, no fixed nodes."""
    m = int(np.ceil(R))
    g = np.stack(np.meshgrid(*(np.arange(-m, m + 1),) * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    g = g[np.linalg.norm(g, axis=1) <= R].astype(np.float64)
    P = (g + jitter * _rng(index, 1).uniform(-1.0, 1.0, g.shape)) * dx
    tri = Delaunay(P)
    tets = tri.simplices.astype(np.int64)
    D = np.stack([P[tets[:, a]] - P[tets[:, 0]] for a in (1, 2, 3)], axis=2)
    tets = tets[np.abs(np.linalg.det(D)) / 6.0 > 1e-6 * dx ** 3]
    hull = np.zeros(P.shape[0], dtype=bool)
    hull[np.unique(tri.convex_hull)] = True
    used = np.zeros(P.shape[0], dtype=bool)
    used[tets.ravel()] = True
    new = -np.ones(P.shape[0], dtype=np.int64)
    new[used] = np.arange(int(used.sum()))
    X = P[used]
    tets = new[tets]
    X[:, 2] += 0.002 - X[:, 2].min()
    n, e = X.shape[0], tets.shape[0]
    v0 = np.array([0.2, 0.0, -0.3])[None, :] + 0.01 * _rng(index, 2).standard_normal((n, 3))
    return TetScene(name=f"unstructured_tet_ball_{e}", X=X, tets=tets, density=1e3,
                    youngs=np.full(e, float(E)), poisson=0.45, corotated=True, volume=True,
                    dirichlet=np.zeros(n, dtype=np.uint8), gravity=np.array([0.0, 0.0, -9.81]), h=0.005,
                    T=T, x0=X.copy(), v0=v0, f_ext=np.zeros((n, 3)),
                    loss_w=_rng(index, 3).standard_normal((n, 3)), tol_fwd=1e-10, tol_bwd=1e-10,
                    k_contact=1e4, mu=0.4, contact=hull[used].astype(np.uint8))
