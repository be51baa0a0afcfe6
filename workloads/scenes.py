"""Scene definitions: seeded synthetic inputs shaped like the paper's beams,
cubes and actuated soft robots (Sec. 6 "Cantilever", Sec. 7 soft robots).

Nothing here depends on the solver.  Each scene is a plain bag of arrays.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Scene:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    origin: np.ndarray                 # (3,) position of grid node (0,0,0)
    cell_mask: Optional[np.ndarray]    # (nx*ny*nz,) uint8 in cell-id order, None = full box
    density: float
    youngs: np.ndarray                 # (e,) Young's modulus per kept cell [Pa]
    poisson: float
    corotated: bool
    volume: bool
    muscle: Optional[np.ndarray]       # (e,) uint8: element carries a muscle fibre energy
    fiber: Optional[np.ndarray]        # (e, 3) unit fibre direction per element
    dirichlet: np.ndarray              # (n,) uint8 per kept node
    contact: np.ndarray                # (n,) uint8 per kept node: penalty-contact candidate
    gravity: np.ndarray                # (3,)
    h: float
    T: int
    x0: np.ndarray                     # (n, 3)
    v0: np.ndarray                     # (n, 3)
    f_ext: np.ndarray                  # (n, 3) constant external force (besides gravity)
    act: Optional[np.ndarray]          # (T, e) contraction signal per step, None = no muscle
    k_contact: float                   # penalty stiffness [N/m] (0 = no contact energy)
    mu: float                          # Coulomb friction coefficient
    loss_w: np.ndarray                 # (n, 3): loss = sum(loss_w * x_T)
    tol_fwd: float
    tol_bwd: float
    # element rule on the kept cells: "hex8" (trilinear hexahedra) or "tet6" (six
    # linear tetrahedra per cell); per-element arrays stay per cell either way
    element_rule: str = "hex8"
    # Neo-Hookean material (Sec. 8): the corotated and volume energies are replaced by
    # the compressible Neo-Hookean energy with mu = w_corot / 2 and lambda = w_vol;
    # A stays the PD matrix of those weights
    neohookean: bool = False

    @property
    def n_nodes(self) -> int:
        return self.x0.shape[0]

    @property
    def n_elems(self) -> int:
        return self.youngs.shape[0]


def grid_node_ids(nx: int, ny: int, nz: int) -> np.ndarray:
    """Grid ids of the 8 corners of every cell, shape (nx*ny*nz, 8).

    Corner a = 4*di + 2*dj + dk addresses node (ci+di, cj+dj, ck+dk)."""
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    out = np.empty((ci.size, 8), dtype=np.int64)
    for a in range(8):
        di, dj, dk = (a >> 2) & 1, (a >> 1) & 1, a & 1
        out[:, a] = ((ci + di) * (ny + 1) + (cj + dj)) * (nz + 1) + (ck + dk)
    return out


def kept_nodes(nx: int, ny: int, nz: int, cell_mask: Optional[np.ndarray]) -> np.ndarray:
    """Sorted grid ids of nodes touched by at least one kept cell."""
    corners = grid_node_ids(nx, ny, nz)
    if cell_mask is not None:
        corners = corners[np.asarray(cell_mask, dtype=bool)]
    return np.unique(corners.ravel())


def _grid_ijk(ids: np.ndarray, ny: int, nz: int):
    k = ids % (nz + 1)
    j = (ids // (nz + 1)) % (ny + 1)
    i = ids // ((nz + 1) * (ny + 1))
    return i, j, k


def _surface_nodes(nx, ny, nz, cell_mask, nodes):
    """1 for kept nodes that touch a missing (or outside) cell."""
    full = np.zeros((nx + 2, ny + 2, nz + 2), dtype=bool)
    if cell_mask is None:
        full[1:-1, 1:-1, 1:-1] = True
    else:
        full[1:-1, 1:-1, 1:-1] = np.asarray(cell_mask, dtype=bool).reshape(nx, ny, nz)
    i, j, k = _grid_ijk(nodes, ny, nz)
    surf = np.zeros(nodes.size, dtype=np.uint8)
    # node (i,j,k) touches padded cells (i+di, j+dj, k+dk), di in {0,1}
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                surf |= (~full[i + di, j + dj, k + dk]).astype(np.uint8)
    return surf


def _rng(scene_index: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(scene_index * 1000 + stream))


def _positions(nx, ny, nz, dx, origin, nodes):
    i, j, k = _grid_ijk(nodes, ny, nz)
    return np.stack([i, j, k], axis=1).astype(np.float64) * dx + np.asarray(origin, np.float64)


def _beam(name, index, nx, ny, nz, dx, E, nu, rho, h, T, *, volume, e_sigma=0.0,
          v0_sigma=0.0, traction=False, tol=1e-9, cell_mask=None):
    nodes = kept_nodes(nx, ny, nz, cell_mask)
    n = nodes.size
    e = int(nx * ny * nz if cell_mask is None else np.count_nonzero(cell_mask))
    i, _, _ = _grid_ijk(nodes, ny, nz)
    dirichlet = (i == 0).astype(np.uint8)
    x0 = _positions(nx, ny, nz, dx, (0.0, 0.0, 0.0), nodes)
    if e_sigma > 0.0:
        youngs = E * np.exp(e_sigma * _rng(index, 1).standard_normal(e))
    else:
        youngs = np.full(e, E, dtype=np.float64)
    v0 = v0_sigma * _rng(index, 2).standard_normal((n, 3)) if v0_sigma > 0 else np.zeros((n, 3))
    v0[dirichlet.astype(bool)] = 0.0
    loss_w = _rng(index, 3).standard_normal((n, 3))
    f_ext = np.zeros((n, 3))
    if traction:
        surf = _surface_nodes(nx, ny, nz, cell_mask, nodes).astype(bool) & ~dirichlet.astype(bool)
        # force scale: 10 % of the weight of one cell of material
        sig = 0.1 * rho * dx ** 3 * 9.81
        f = sig * _rng(index, 4).standard_normal((n, 3))
        f_ext[surf] = f[surf]
    return Scene(name=name, nx=nx, ny=ny, nz=nz, dx=dx, origin=np.zeros(3), cell_mask=cell_mask,
                 density=rho, youngs=youngs, poisson=nu, corotated=True, volume=volume,
                 muscle=None, fiber=None, dirichlet=dirichlet,
                 contact=np.zeros(n, dtype=np.uint8), gravity=np.array([0.0, 0.0, -9.81]),
                 h=h, T=T, x0=x0, v0=v0, f_ext=f_ext, act=None, k_contact=0.0, mu=0.0,
                 loss_w=loss_w, tol_fwd=tol, tol_bwd=tol)


def neohookean_beam(nx=5, ny=3, nz=4, *, T=6, index=9, E=1e5, twist=0.0) -> Scene:
    """Small cantilever of the Neo-Hookean material (Sec. 8): the small beam with
    the corotated and volume weights read as (2 mu, lambda), seeded stiffness
    variation and tractions; `twist` adds an initial angular velocity [rad/s] about
    the beam axis (large rotations within a few steps)."""
    sc = _beam(f"neohookean_beam_{nx}x{ny}x{nz}", index, nx, ny, nz, 0.01, E, 0.45, 1e3, 0.01, T,
               volume=True, e_sigma=0.2, v0_sigma=0.01, traction=True, tol=1e-10)
    if twist != 0.0:
        c = sc.x0.mean(axis=0)
        r = sc.x0 - c
        w = np.array([twist, 0.0, 0.0])
        v = np.cross(w[None, :], r)
        v[sc.dirichlet.astype(bool)] = 0.0
        sc.v0 = sc.v0 + v
    sc.neohookean = True
    return sc


def cantilever_c1(T: int = 50) -> Scene:
    """4x4x8-cell cantilever (225 nodes, 675 DoFs), x=0 face fixed, gravity,
    corotated energy E=1e5, nu=0.45, rho=1e3, h=0.01, v0 ~ N(0, 0.01^2)."""
    return _beam("c1_cantilever_4x4x8", 1, 8, 4, 4, 0.01, 1e5, 0.45, 1e3, 0.01, T,
                 volume=False, v0_sigma=0.01, tol=1e-9)


def beam_c2(T: int = 100) -> Scene:
    """32x32x64-cell beam (70,785 nodes), corotated + volume, E lognormal(1e6, 0.2)."""
    return _beam("c2_beam_32x32x64", 2, 64, 32, 32, 0.01, 1e6, 0.45, 1e3, 0.01, T,
                 volume=True, e_sigma=0.2, tol=1e-8)


def beam_c5(T: int = 500) -> Scene:
    """64x64x128-cell beam (545,025 nodes), corotated, gravity + surface tractions."""
    return _beam("c5_beam_64x64x128", 5, 128, 64, 64, 0.01, 1e6, 0.45, 1e3, 0.01, T,
                 volume=False, traction=True, tol=1e-8)


def small_beam(nx=4, ny=2, nz=2, *, T=5, volume=True, index=7, E=1e5, e_sigma=0.2,
               v0_sigma=0.01, traction=True, tol=1e-10) -> Scene:
    """Small beam used by the parity tests (ragged sizes, several supernodes)."""
    return _beam(f"small_beam_{nx}x{ny}x{nz}", index, nx, ny, nz, 0.01, E, 0.45, 1e3, 0.01, T,
                 volume=volume, e_sigma=e_sigma, v0_sigma=v0_sigma, traction=traction, tol=tol)


def contact_cube_c3(N: int = 24, T: int = 200, index: int = 3) -> Scene:
    """N^3-cell cube dropped from 0.05 m onto the ground z=0 with penalty
    contact (k=1e4 N/m on every surface node) and Coulomb friction mu=0.5."""
    nx = ny = nz = N
    dx = 0.01
    nodes = kept_nodes(nx, ny, nz, None)
    n = nodes.size
    origin = np.array([0.0, 0.0, 0.05])
    x0 = _positions(nx, ny, nz, dx, origin, nodes)
    contact = _surface_nodes(nx, ny, nz, None, nodes)
    v0 = 0.1 * _rng(index, 2).standard_normal((n, 3))
    return Scene(name=f"c3_contact_cube_{N}", nx=nx, ny=ny, nz=nz, dx=dx, origin=origin,
                 cell_mask=None, density=1e3, youngs=np.full(N ** 3, 1e6), poisson=0.45,
                 corotated=True, volume=True, muscle=None, fiber=None,
                 dirichlet=np.zeros(n, dtype=np.uint8), contact=contact,
                 gravity=np.array([0.0, 0.0, -9.81]), h=0.005, T=T, x0=x0, v0=v0,
                 f_ext=np.zeros((n, 3)), act=None, k_contact=1e4, mu=0.5,
                 loss_w=_rng(index, 3).standard_normal((n, 3)), tol_fwd=1e-8, tol_bwd=1e-8)


def quadruped_mask(N: int) -> np.ndarray:
    """Quadruped template in an N^3 box: body = top ceil(N/2) layers, legs =
    four ceil(N/4) x ceil(N/4) corner columns below it (cell-id order)."""
    body = int(math.ceil(N / 2))
    leg = int(math.ceil(N / 4))
    m = np.zeros((N, N, N), dtype=np.uint8)
    m[:, :, N - body:] = 1
    for lo_i in (0, N - leg):
        for lo_j in (0, N - leg):
            m[lo_i:lo_i + leg, lo_j:lo_j + leg, :N - body] = 1
    return m.ravel()


def quadruped(N: int, T: int = 100, index: int = 4, request: int = 0) -> Scene:
    """Actuated soft quadruped (C4 request): legs carry z-fibres with
    contraction a_e(t) ~ U[0, 0.3]; feet rest on the ground z=0."""
    nx = ny = nz = N
    dx = 0.01
    mask = quadruped_mask(N)
    nodes = kept_nodes(nx, ny, nz, mask)
    n = nodes.size
    e = int(np.count_nonzero(mask))
    cells = np.flatnonzero(mask)
    ck = cells % nz
    body = int(math.ceil(N / 2))
    leg_el = (ck < N - body).astype(np.uint8)
    fiber = np.zeros((e, 3))
    fiber[:, 2] = 1.0
    rng_seed = index * 100 + request
    act = _rng(rng_seed, 5).uniform(0.0, 0.3, size=(T, e)) * leg_el[None, :]
    x0 = _positions(nx, ny, nz, dx, (0.0, 0.0, 0.0), nodes)
    contact = _surface_nodes(nx, ny, nz, mask, nodes)
    v0 = 0.01 * _rng(rng_seed, 2).standard_normal((n, 3))
    return Scene(name=f"c4_quadruped_{N}", nx=nx, ny=ny, nz=nz, dx=dx, origin=np.zeros(3),
                 cell_mask=mask, density=1e3, youngs=np.full(e, 1e6), poisson=0.45,
                 corotated=True, volume=True, muscle=leg_el, fiber=fiber,
                 dirichlet=np.zeros(n, dtype=np.uint8), contact=contact,
                 gravity=np.array([0.0, 0.0, -9.81]), h=0.01, T=T, x0=x0, v0=v0,
                 f_ext=np.zeros((n, 3)), act=act, k_contact=1e4, mu=0.5,
                 loss_w=_rng(rng_seed, 3).standard_normal((n, 3)), tol_fwd=1e-8, tol_bwd=1e-8)


def serving_stream_c4(n_requests: int = 256, rate_hz: float = 50.0, T: int = 100,
                      n_min: int = 8, n_max: int = 24, index: int = 4):
    """Poisson request stream: exponential inter-arrival times at `rate_hz`
    and request sizes N ~ U{n_min..n_max}.  Returns (arrival_s, sizes)."""
    rng = _rng(index, 6)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    sizes = rng.integers(n_min, n_max + 1, size=n_requests)
    return np.cumsum(gaps) - gaps[0], sizes


def _sphere_mask(D: int, R: float) -> np.ndarray:
    c = np.arange(D) + 0.5
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    return (((X - D / 2) ** 2 + (Y - D / 2) ** 2 + (Z - D / 2) ** 2) <= R * R).astype(np.uint8).ravel()


def rolling_sphere(T: int = 100, v: float = 0.2, index: int = 6) -> Scene:
    """Soft sphere rolling on the ground z = 0 with complementarity contact: the
    cells of a 10^3 grid whose centres lie within 5 cells of its centre (552
    elements, 823 nodes = 2469 DoFs, the paper's rolling-sphere size), dx = 1 cm,
    resting on the ground and rolling along +x without slipping (v_x = v,
    omega_y = v / radius).  Contact candidates: the 72 surface nodes of the lower
    front quarter in a 5-node band around the rolling plane (|y - y_c| <= 2 dx,
    z <= z_c, x >= x_c - dx), the region the rolling brings down to the ground."""
    D, dx = 10, 0.01
    mask = _sphere_mask(D, 5.0)
    nodes = kept_nodes(D, D, D, mask)
    n = nodes.size
    e = int(np.count_nonzero(mask))
    i, j, k = _grid_ijk(nodes, D, D)
    x0 = _positions(D, D, D, dx, (0.0, 0.0, 0.0), nodes)
    surf = _surface_nodes(D, D, D, mask, nodes).astype(bool)
    contact = (surf & (np.abs(j - 5) <= 2) & (k <= 5) & (i >= 4)).astype(np.uint8)
    centre = np.full(3, 5 * dx)
    radius = 5 * dx
    omega = np.array([0.0, v / radius, 0.0])
    v0 = np.array([v, 0.0, 0.0])[None, :] + np.cross(omega[None, :], x0 - centre[None, :])
    return Scene(name="rolling_sphere", nx=D, ny=D, nz=D, dx=dx, origin=np.zeros(3), cell_mask=mask,
                 density=1e3, youngs=np.full(e, 1e5), poisson=0.45, corotated=True, volume=True,
                 muscle=None, fiber=None, dirichlet=np.zeros(n, dtype=np.uint8), contact=contact,
                 gravity=np.array([0.0, 0.0, -9.81]), h=0.005, T=T, x0=x0, v0=v0, f_ext=np.zeros((n, 3)),
                 act=None, k_contact=0.0, mu=0.0, loss_w=_rng(index, 3).standard_normal((n, 3)),
                 tol_fwd=1e-6, tol_bwd=1e-6)


def napkin(N: int, frac: float, T: int = 3, gap: float = 5e-4, v_drop: float = 0.2, index: int = 7) -> Scene:
    """One-layer N x N x 1-cell napkin (2 (N+1)^2 nodes; N = 25 ... 100 gives the
    paper's 4056 ... 61206 DoFs), dx = 1 cm, gap above the ground z = 0.  The
    nodes over a central disc move down at v_drop, so the disc's bottom nodes
    reach the ground in the first step; the disc holds round(frac * n) bottom
    nodes (frac <= 0.5: at most every bottom node), which sets the contact-set
    size as the obstacle's solid angle does in the paper.  Candidates: every
    bottom node."""
    nx = ny = N
    nz = 1
    dx = 0.01
    nodes = kept_nodes(nx, ny, nz, None)
    n = nodes.size
    i, j, k = _grid_ijk(nodes, ny, nz)
    x0 = _positions(nx, ny, nz, dx, (0.0, 0.0, gap), nodes)
    bottom = k == 0
    # disc: the round(frac * n) bottom nodes nearest the centre (ties by node order)
    r2 = (i - N / 2) ** 2 + (j - N / 2) ** 2
    want = min(int(round(frac * n)), int(bottom.sum()))
    order = np.lexsort((np.arange(n), r2))
    order = order[bottom[order]][:want]
    disc_ij = set(zip(i[order].tolist(), j[order].tolist()))
    in_disc = np.array([(a, b) in disc_ij for a, b in zip(i.tolist(), j.tolist())])
    v0 = np.zeros((n, 3))
    v0[in_disc, 2] = -v_drop
    return Scene(name=f"napkin_{N}x{N}x1_{int(round(100 * frac))}", nx=nx, ny=ny, nz=nz, dx=dx,
                 origin=np.array([0.0, 0.0, gap]), cell_mask=None, density=1e3, youngs=np.full(N * N, 1e5),
                 poisson=0.45, corotated=True, volume=True, muscle=None, fiber=None,
                 dirichlet=np.zeros(n, dtype=np.uint8), contact=bottom.astype(np.uint8),
                 gravity=np.array([0.0, 0.0, -9.81]), h=0.005, T=T, x0=x0, v0=v0, f_ext=np.zeros((n, 3)),
                 act=None, k_contact=0.0, mu=0.0, loss_w=_rng(index, 3).standard_normal((n, 3)),
                 tol_fwd=1e-6, tol_bwd=1e-6)


SCENES = {
    "c1": cantilever_c1,
    "c2": beam_c2,
    "c3": contact_cube_c3,
    "c5": beam_c5,
}


def tet_beam(nx=4, ny=2, nz=2, *, T=5, **kw) -> Scene:
    """small_beam meshed with six tetrahedra per cell (tet6 rule); materials,
    boundary, loads and loss weights as the hexahedral beam."""
    sc = small_beam(nx, ny, nz, T=T, **kw)
    return dataclasses.replace(sc, name=f"tet_beam_{nx}x{ny}x{nz}", element_rule="tet6")


def tet_ball(T: int = 20, index: int = 8) -> Scene:
    """Ball of 336 linear tetrahedra: the cells of a 6^3 grid within 2.4 cells of
    its centre, six tetrahedra each (117 nodes, 351 DoFs; the paper's tennis-ball
    mesh has 320 tetrahedra, Sec. 7), dx = 1 cm, its lowest nodes 2 mm above the
    ground z = 0, moving at (0.2, 0, -0.3) m/s plus N(0, 0.01^2) per DoF; penalty
    contact k = 1e4 N/m on the surface nodes with Coulomb friction mu = 0.4."""
    D, dx = 6, 0.01
    mask = _sphere_mask(D, 2.4)
    nodes = kept_nodes(D, D, D, mask)
    n = nodes.size
    e = int(np.count_nonzero(mask))
    i, j, k = _grid_ijk(nodes, D, D)
    origin = np.array([0.0, 0.0, 0.002 - dx * float(k.min())])
    x0 = _positions(D, D, D, dx, origin, nodes)
    contact = _surface_nodes(D, D, D, mask, nodes)
    v0 = np.array([0.2, 0.0, -0.3])[None, :] + 0.01 * _rng(index, 2).standard_normal((n, 3))
    return Scene(name="tet_ball_336", nx=D, ny=D, nz=D, dx=dx, origin=origin, cell_mask=mask,
                 density=1e3, youngs=np.full(e, 1e5), poisson=0.45, corotated=True, volume=True,
                 muscle=None, fiber=None, dirichlet=np.zeros(n, dtype=np.uint8), contact=contact,
                 gravity=np.array([0.0, 0.0, -9.81]), h=0.005, T=T, x0=x0, v0=v0,
                 f_ext=np.zeros((n, 3)), act=None, k_contact=1e4, mu=0.4,
                 loss_w=_rng(index, 3).standard_normal((n, 3)), tol_fwd=1e-10, tol_bwd=1e-10,
                 element_rule="tet6")
