"""Pins for the oracle's tetrahedral rule (six linear tetrahedra per voxel cell,
one point each; the paper's tetrahedral meshes, Secs. 5.1 and 7, are not
available, so voxel-built tetrahedra stand in): shape-function identities and
the affine patch test, a conforming split, volumes and lumped mass, the
structure of A (Eqn 19), the rest / translation / rotation invariants, the PD
fixed point equal to Newton's, and central finite differences of every gradient
block through contact, friction and muscles."""
import dataclasses
from collections import Counter

import numpy as np

from oracle import adjoint, newton, pd_cpu
from oracle.mesh import VoxelMesh, kuhn_tetrahedra
from oracle.model import Model
from test_oracle_dynamics import _loss, tiny_everything_scene
from workloads import tet_ball, tet_beam


def _mesh(sc):
    return VoxelMesh(sc.nx, sc.ny, sc.nz, sc.dx, sc.origin, sc.cell_mask, rule="tet6")


def test_tet_shape_functions_partition_and_patch_test():
    sc = tet_beam(3, 2, 2)
    mesh = _mesh(sc)
    assert mesh.gradN.shape == (6, 8, 3)
    # partition of unity: sum_a grad N_a = 0 at every point
    assert np.max(np.abs(mesh.gradN.sum(axis=1))) < 1e-12 / sc.dx
    # each tetrahedron touches exactly its 4 corners
    for q, tet in enumerate(kuhn_tetrahedra()):
        nz = set(np.flatnonzero(np.abs(mesh.gradN[q]).sum(axis=1)).tolist())
        assert nz == set(tet)
    # affine patch test: x = A X + b gives F = A exactly at every point
    rng = np.random.default_rng(1)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    x = mesh.X @ A.T + rng.standard_normal(3)
    F = mesh.deformation_gradients(x)
    assert F.shape == (mesh.e, 6, 3, 3)
    assert np.max(np.abs(F - A[None, None])) < 1e-12


def test_tet_split_is_conforming():
    """Every interior triangle is shared by exactly two tetrahedra (of the same or
    neighbouring cells); the others lie on the boundary of the box."""
    sc = tet_beam(3, 2, 2)
    mesh = _mesh(sc)
    faces = Counter()
    for tet in kuhn_tetrahedra():
        for drop in range(4):
            tri = [tet[i] for i in range(4) if i != drop]
            for e in range(mesh.e):
                faces[tuple(sorted(mesh.elems[e, tri].tolist()))] += 1
    lo, hi = mesh.X.min(axis=0), mesh.X.max(axis=0)
    for tri, cnt in faces.items():
        assert cnt in (1, 2)
        if cnt == 1:
            P = mesh.X[list(tri)]
            on = [np.allclose(P[:, d], lo[d]) or np.allclose(P[:, d], hi[d]) for d in range(3)]
            assert any(on), tri


def test_tet_volumes_and_lumped_mass():
    for sc in (tet_beam(3, 2, 2), tet_ball(T=1)):
        mesh = _mesh(sc)
        assert np.isclose(6 * mesh.Vq, sc.dx ** 3, rtol=1e-14)
        m = mesh.lumped_mass(sc.density)
        assert np.isclose(m.sum(), sc.density * mesh.e * sc.dx ** 3, rtol=1e-13)
    # one cell: the two diagonal corners carry rho dx^3 / 4, the other six rho dx^3 / 12
    mesh = VoxelMesh(1, 1, 1, 0.01, rule="tet6")
    m = mesh.lumped_mass(1e3)
    corner = 1e3 * 1e-6
    expect = np.full(8, corner / 12)
    expect[[0, 7]] = corner / 4
    assert np.allclose(m[mesh.elems[0]], expect, rtol=1e-13)


def test_tet_A_is_kron_I3_LA_and_rows_sum_to_mass():
    sc = tet_beam(3, 2, 2)
    model = Model(sc)
    A = model.A_matrix().toarray()
    LA = A[0::3, 0::3]
    for i in range(3):
        for j in range(3):
            blk = A[i::3, j::3]
            if i == j:
                assert np.allclose(blk, LA, atol=0)
            else:
                assert np.max(np.abs(blk)) == 0.0
    assert np.allclose(LA.sum(axis=1), model.m / model.h ** 2, rtol=1e-12)
    # the tetrahedral stencil differs from the hexahedral one
    Ah = Model(dataclasses.replace(sc, element_rule="hex8")).A_matrix().toarray()
    assert np.max(np.abs(A - Ah)) > 1e-3 * np.max(np.abs(Ah))


def test_tet_rest_translation_rotation_invariants():
    base = tet_beam(3, 2, 2, T=3)
    n = base.x0.shape[0]
    free = dict(dirichlet=np.zeros(n, dtype=np.uint8), gravity=np.zeros(3), f_ext=np.zeros((n, 3)))
    # rest stays at rest
    sc = dataclasses.replace(base, v0=np.zeros((n, 3)), **free)
    m = Model(sc)
    xs, _, _ = newton.rollout(m, sc.x0, sc.v0, sc.f_ext)
    assert np.max(np.abs(xs - sc.x0[None])) < 1e-14
    # uniform translation is exact
    v = np.array([0.1, -0.2, 0.05])
    sc = dataclasses.replace(base, v0=np.tile(v, (n, 1)), **free)
    m = Model(sc)
    xs, _, _ = newton.rollout(m, sc.x0, sc.v0, sc.f_ext)
    for t in range(xs.shape[0]):
        assert np.max(np.abs(xs[t] - (sc.x0 + t * sc.h * v))) < 1e-13
    # a rigidly rotated rest mesh stays put
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    x0 = sc.x0 @ Q.T
    sc = dataclasses.replace(base, x0=x0, v0=np.zeros((n, 3)), **free)
    m = Model(sc)
    xs, _, _ = newton.rollout(m, x0, sc.v0, sc.f_ext)
    assert np.max(np.abs(xs - x0[None])) < 1e-12


def test_tet_pd_fixed_point_equals_newton():
    sc = tet_beam(4, 2, 2, T=3)
    m = Model(sc)
    xs, _, infos = newton.rollout(m, sc.x0, sc.v0, sc.f_ext)
    for info in infos:
        assert info["residual"] <= 1e-12 * info["ref"]
    xp, _, _ = pd_cpu.rollout(m, sc.x0, sc.v0, sc.f_ext)
    assert np.max(np.abs(xp - xs)) < 1e-10


def test_tet_gradients_match_central_fd_everything():
    sc = dataclasses.replace(tiny_everything_scene(), element_rule="tet6")
    m = Model(sc)
    xs, vs, _ = newton.rollout(m, sc.x0, sc.v0, sc.f_ext, sc.act)
    assert np.any(xs[:-1][:, m.contact, 2] < 0)
    _, gx = adjoint.final_position_loss(m, xs, sc.loss_w)
    g = adjoint.backward(m, xs, vs, gx, act=sc.act)
    gE, gnu = adjoint.material_gradients(m, g)
    rng = np.random.default_rng(13)

    def fd(fun, eps):
        return (fun(eps) - fun(-eps)) / (2 * eps)

    checks = []
    d = rng.standard_normal(sc.x0.shape)
    checks.append((fd(lambda s: _loss(sc, x0=sc.x0 + s * d), 1e-7), np.sum(g["g_x0"] * d)))
    checks.append((fd(lambda s: _loss(sc, v0=sc.v0 + s * d), 1e-6), np.sum(g["g_v0"] * d)))
    checks.append((fd(lambda s: _loss(sc, f_ext=sc.f_ext + s * d), 1e-6), np.sum(g["g_fext"] * d)))
    dE = rng.standard_normal(m.mesh.e) * sc.youngs
    checks.append((fd(lambda s: _loss(sc, youngs=sc.youngs + s * dE), 1e-6), np.sum(gE * dE)))
    checks.append((fd(lambda s: _loss(sc, poisson=sc.poisson + s), 1e-6), gnu))
    checks.append((fd(lambda s: _loss(sc, mu=sc.mu + s), 1e-6), g["g_mu"]))
    da = rng.standard_normal(sc.act.shape)
    checks.append((fd(lambda s: _loss(sc, act=sc.act + s * da), 1e-6), np.sum(g["g_act"] * da)))
    for num, ana in checks:
        assert abs(num - ana) <= 2e-6 * max(abs(num), 1e-12), (num, ana)
