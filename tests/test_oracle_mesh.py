"""Pins for the oracle's discretisation: closed forms of the trilinear hex
element (partition of unity, affine patch test), mass, and the structure
A = I_3 (x) L_A of the PD matrix (Eqn 19)."""
import numpy as np
import scipy.sparse as sp

from oracle.mesh import VoxelMesh, shape_gradients
from oracle.model import Model
from workloads import cantilever_c1, small_beam, quadruped


def test_partition_of_unity_gradients():
    g = shape_gradients(0.01)
    assert np.allclose(g.sum(axis=1), 0.0, atol=1e-12)


def test_affine_patch_test_F_exact():
    """For x = B X + c the deformation gradient is B at every Gauss point."""
    mesh = VoxelMesh(3, 2, 2, 0.01)
    rng = np.random.default_rng(0)
    B = rng.standard_normal((3, 3))
    c = rng.standard_normal(3)
    x = mesh.X @ B.T + c
    F = mesh.deformation_gradients(x)
    assert np.allclose(F, B[None, None], atol=1e-12)


def test_G_matrix_matches_F():
    mesh = VoxelMesh(2, 1, 1, 0.02)
    rng = np.random.default_rng(1)
    x = mesh.X + 1e-3 * rng.standard_normal(mesh.X.shape)
    F = mesh.deformation_gradients(x)
    G = mesh.G_matrix()
    for e in range(mesh.e):
        xe = x[mesh.elems[e]].ravel()
        for q in range(8):
            assert np.allclose(G[q] @ xe, F[e, q].ravel(), atol=1e-13)


def test_total_mass_equals_rho_volume():
    for sc in (cantilever_c1(), quadruped(8, T=1)):
        mesh = VoxelMesh(sc.nx, sc.ny, sc.nz, sc.dx, sc.origin, sc.cell_mask)
        m = mesh.lumped_mass(sc.density)
        assert np.isclose(m.sum(), sc.density * mesh.e * sc.dx ** 3, rtol=1e-14)


def test_A_is_kron_I3_LA_and_rows_sum_to_mass():
    sc = small_beam(3, 2, 2)
    model = Model(sc)
    A = model.A_matrix().toarray()
    n = model.mesh.n
    LA = A[0::3, 0::3]
    for i in range(3):
        for j in range(3):
            blk = A[i::3, j::3]
            if i == j:
                assert np.allclose(blk, LA, atol=0)
            else:
                assert np.max(np.abs(blk)) == 0.0
    # constants are in the null space of sum w G^T G: row sums = m/h^2
    assert np.allclose(LA.sum(axis=1), model.m / model.h ** 2, rtol=1e-12)
    assert LA.shape == (n, n)


def test_affine_interior_force_vanishes():
    """A constant stress field exerts no net force on interior nodes."""
    sc = small_beam(4, 4, 4, traction=False, e_sigma=0.0)
    model = Model(sc)
    A = model.A_matrix()
    M = sp.diags(np.repeat(model.m / model.h ** 2, 3))
    K = (A - M).toarray()
    rng = np.random.default_rng(2)
    B = rng.standard_normal((3, 3))
    x = (model.mesh.X @ B.T).ravel()
    f = (K @ x).reshape(-1, 3)
    ijk = model.mesh.ijk
    interior = np.all((ijk > 0) & (ijk < np.array([sc.nx, sc.ny, sc.nz])), axis=1)
    assert interior.any()
    assert np.max(np.abs(f[interior])) < 1e-9 * np.max(np.abs(f))


def test_affine_energy_closed_form():
    """E(B X) = w/2 * volume * |B - R(B)|^2 for a homogeneous deformation."""
    sc = small_beam(2, 2, 2, volume=False, e_sigma=0.0, traction=False)
    model = Model(sc)
    rng = np.random.default_rng(3)
    B = np.eye(3) + 0.1 * rng.standard_normal((3, 3))
    U, s, Vt = np.linalg.svd(B)
    R = U @ Vt
    x = model.mesh.X @ B.T
    vol = model.mesh.e * sc.dx ** 3
    expect = 0.5 * model.w_corot[0] * vol * np.sum((B - R) ** 2)
    assert np.isclose(model.energy(x), expect, rtol=1e-12)
