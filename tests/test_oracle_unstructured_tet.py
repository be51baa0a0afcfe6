"""Pins for the oracle's unstructured tetrahedral meshes (oracle/tetmesh.py,
oracle/tetstructure.py; Secs. 5.1 and 7 use tetrahedral meshes with their own node
sets): partition of unity of the shape functions, the affine patch test, volumes
that tile the box and the lumped mass, rest and rigid-motion invariants, the
gradient and Hessian against central differences, the PD + L-BFGS fixed point
against Newton's, the adjoint against differences of a rollout loss, and the graph
nested dissection (a permutation whose separators disconnect their two sides, and a
supernodal structure that holds the exact Cholesky fill of L_A)."""
import numpy as np
import pytest

from oracle import adjoint, newton, pd_cpu
from oracle.tetmesh import TetModel
from oracle.tetstructure import analyse, free_adjacency
from workloads import unstructured_tet_beam


@pytest.fixture(scope="module")
def beam():
    return unstructured_tet_beam(6, 3, 3, T=2)


def _rot(rng):
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    return Q


def test_shape_functions_volumes_and_mass(beam):
    m = TetModel(beam)
    g = m.mesh.gradN[:, 0]
    assert np.abs(g.sum(axis=1)).max() <= 1e-9 * np.abs(g).max()          # partition of unity
    rng = np.random.default_rng(1)
    A = np.eye(3) + 0.1 * rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    F = m.mesh.deformation_gradients(beam.X @ A.T + b)
    assert np.abs(F - A[None, None]).max() <= 1e-10                         # affine patch test
    box = 6 * 3 * 3 * 0.01 ** 3
    assert abs(m.mesh.Vq.sum() - box) <= 1e-12 * box                        # the tetrahedra tile the box
    assert abs(m.m.sum() - beam.density * box) <= 1e-12 * beam.density * box


def test_rest_and_rigid_motions_are_stress_free(beam):
    m = TetModel(beam)
    assert abs(m.energy(beam.X)) <= 1e-20
    assert np.abs(m.grad_E(beam.X)).max() <= 1e-12
    rng = np.random.default_rng(2)
    x = beam.X @ _rot(rng).T + rng.standard_normal(3)
    assert abs(m.energy(x)) <= 1e-18
    assert np.abs(m.grad_E(x)).max() <= 1e-9


def test_gradient_and_hessian_match_differences(beam):
    m = TetModel(beam)
    rng = np.random.default_rng(3)
    x = beam.X + 0.1 * 0.01 * rng.standard_normal(beam.X.shape)
    g = m.grad_E(x)
    d = rng.standard_normal(x.shape)
    eps = 1e-7
    fd = (m.energy(x + eps * d) - m.energy(x - eps * d)) / (2 * eps)
    assert abs(fd - np.sum(g * d)) <= 1e-6 * abs(fd)
    H = m.hessian(x)
    Hd = (H @ d.ravel()).reshape(x.shape) - (m.m / m.h ** 2)[:, None] * d
    fdg = (m.grad_E(x + eps * d) - m.grad_E(x - eps * d)) / (2 * eps)
    assert np.abs(fdg - Hd).max() <= 1e-5 * np.abs(Hd).max()


def test_pd_lbfgs_reaches_the_newton_fixed_point(beam):
    m = TetModel(beam)
    xn, _, _ = newton.newton_step(m, beam.x0, beam.v0, beam.f_ext)
    xp, _, _ = pd_cpu.pd_lbfgs_step(m, pd_cpu.ScalarA(m), beam.x0, beam.v0, beam.f_ext, None, None, 1e-12, 5, 5000)
    assert np.linalg.norm(xp - xn) <= 1e-9 * np.linalg.norm(xn - beam.x0)


def test_adjoint_matches_central_differences(beam):
    m = TetModel(beam)
    xs, vs, _ = newton.rollout(m, beam.x0, beam.v0, beam.f_ext, T=beam.T)
    _, gx = adjoint.final_position_loss(m, xs, beam.loss_w)
    g = adjoint.backward(m, xs, vs, gx)
    rng = np.random.default_rng(4)
    d = rng.standard_normal(beam.x0.shape)
    d[m.dirichlet] = 0.0

    def loss(v0=None, f=None, E=None):
        mm = TetModel(beam, youngs=E)
        out, _, _ = newton.rollout(mm, beam.x0, beam.v0 if v0 is None else v0,
                                   beam.f_ext if f is None else f, T=beam.T)
        return float(np.sum(beam.loss_w * out[-1]))
    eps = 1e-6
    fd_v = (loss(v0=beam.v0 + eps * d) - loss(v0=beam.v0 - eps * d)) / (2 * eps)
    assert abs(fd_v - np.sum(g["g_v0"] * d)) <= 2e-6 * abs(fd_v)
    fd_f = (loss(f=beam.f_ext + eps * d) - loss(f=beam.f_ext - eps * d)) / (2 * eps)
    assert abs(fd_f - np.sum(g["g_fext"] * d)) <= 2e-6 * abs(fd_f)
    gE, _ = adjoint.material_gradients(m, g)
    dE = rng.standard_normal(m.mesh.e) * beam.youngs
    fd_E = (loss(E=beam.youngs + eps * dE) - loss(E=beam.youngs - eps * dE)) / (2 * eps)
    assert abs(fd_E - np.sum(gE * dE)) <= 2e-6 * abs(fd_E)


@pytest.mark.parametrize("leaf", [8, 16, 64])
def test_graph_nested_dissection(leaf):
    sc = unstructured_tet_beam(8, 4, 4, T=1)
    st = analyse(sc.X, sc.tets, sc.dirichlet, leaf_max=leaf)
    perm, first = st["perm"], st["snode_first"]
    free, adj = free_adjacency(sc.tets, sc.dirichlet)
    assert np.array_equal(np.sort(perm), np.arange(free.size))              # a permutation of the free nodes
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    # every supernode's nodes are adjacent (in the permuted numbering) only to nodes
    # of its own subtree or of its ancestors: the elimination tree is a tree
    ns = first.size - 1
    owner = np.repeat(np.arange(ns), np.diff(first))
    parent = st["parent"]

    def ancestors(s):
        out = set()
        while s >= 0:
            out.add(int(s))
            s = int(parent[s])
        return out
    anc = [ancestors(s) for s in range(ns)]
    for k in range(perm.size):
        for j in st["adj"][k]:
            a, b = int(owner[k]), int(owner[j])
            assert a in anc[b] or b in anc[a], (a, b)
    # the exact Cholesky factor of L_A (x block of A on the free DoFs, permuted) has
    # its nonzeros inside the supernodal row structure
    m = TetModel(sc)
    A = m.A_matrix().toarray()[np.ix_(m.free_dofs[0::3], m.free_dofs[0::3])]
    Ap = A[np.ix_(perm, perm)]
    L = np.linalg.cholesky(Ap)
    rows, rp = st["rows"], st["row_ptr"]
    allowed = np.zeros_like(L, dtype=bool)
    for s in range(ns):
        r = rows[rp[s]:rp[s + 1]]
        for c in range(first[s], first[s + 1]):
            allowed[r[r >= c], c] = True
    assert np.abs(L[~allowed]).max(initial=0.0) <= 1e-12 * np.abs(L).max()


def test_voxel_split_agrees_with_the_voxel_rule():
    """A voxel beam split six ways, handed to the unstructured model as a plain list
    of tetrahedra (its nodes, the cells' Kuhn tetrahedra, each cell's Young's modulus
    on its six tetrahedra), is the same discretisation as the voxel model's tet6
    rule: same lumped mass, energy, forces, Hessian and A, and per-tetrahedron
    material gradients that add up to the per-cell ones."""
    from oracle.mesh import kuhn_tetrahedra
    from oracle.model import Model
    from workloads import TetScene, tet_beam
    sv = tet_beam(4, 3, 2, T=2)
    mv = Model(sv)
    kt = np.array(kuhn_tetrahedra())
    tets = mv.mesh.elems[:, kt].reshape(-1, 4)
    st = TetScene(name="split", X=mv.mesh.X, tets=tets, density=sv.density,
                  youngs=np.repeat(sv.youngs, 6), poisson=sv.poisson, corotated=sv.corotated,
                  volume=sv.volume, dirichlet=sv.dirichlet, gravity=sv.gravity, h=sv.h, T=sv.T,
                  x0=sv.x0, v0=sv.v0, f_ext=sv.f_ext, loss_w=sv.loss_w, tol_fwd=sv.tol_fwd,
                  tol_bwd=sv.tol_bwd)
    mt = TetModel(st)
    assert np.allclose(mt.m, mv.m, rtol=1e-13, atol=0)
    rng = np.random.default_rng(5)
    x = sv.x0 + 0.02 * sv.dx * rng.standard_normal(sv.x0.shape)
    assert abs(mt.energy(x) - mv.energy(x)) <= 1e-12 * abs(mv.energy(x))
    g = mv.grad_E(x)
    assert np.abs(mt.grad_E(x) - g).max() <= 1e-11 * np.abs(g).max()
    Hv, Ht = mv.hessian(x).toarray(), mt.hessian(x).toarray()
    assert np.abs(Ht - Hv).max() <= 1e-11 * np.abs(Hv).max()
    Av, At = mv.A_matrix().toarray(), mt.A_matrix().toarray()
    assert np.abs(At - Av).max() <= 1e-12 * np.abs(Av).max()
    xs, vs, _ = newton.rollout(mv, sv.x0, sv.v0, sv.f_ext, T=sv.T)
    _, gx = adjoint.final_position_loss(mv, xs, sv.loss_w)
    gv = adjoint.backward(mv, xs, vs, gx)
    gt = adjoint.backward(mt, xs, vs, gx)
    for k in ("g_wc", "g_wv"):
        cell = gt[k].reshape(-1, 6).sum(axis=1)
        assert np.abs(cell - gv[k]).max() <= 1e-9 * np.abs(gv[k]).max(), k
    assert np.abs(gt["g_v0"] - gv["g_v0"]).max() <= 1e-9 * np.abs(gv["g_v0"]).max()


@pytest.fixture(scope="module")
def nh_beam():
    import dataclasses
    return dataclasses.replace(unstructured_tet_beam(6, 3, 3, T=2), neohookean=True)


def test_neohookean_rest_rigid_and_derivatives(nh_beam):
    """Neo-Hookean tetrahedra (the paper's Armadillo): stress-free at rest and under
    rigid motions, gradient and Hessian against central differences."""
    m = TetModel(nh_beam)
    X = nh_beam.X
    scale = np.sum(m.nh_mu * m.mesh.Vq)                  # energy of a unit strain, roughly
    fscale = scale / 0.01                                # force of a unit strain at dx = 1 cm
    assert abs(m.energy(X)) <= 1e-14 * scale and np.abs(m.grad_E(X)).max() <= 1e-12 * fscale
    rng = np.random.default_rng(8)
    xr = X @ _rot(rng).T + rng.standard_normal(3)
    assert abs(m.energy(xr)) <= 1e-12 * scale and np.abs(m.grad_E(xr)).max() <= 1e-10 * fscale
    x = X + 0.01 * 0.01 * rng.standard_normal(X.shape)
    assert np.linalg.det(m.mesh.deformation_gradients(x)[:, 0]).min() > 0.25
    g = m.grad_E(x)
    d = rng.standard_normal(X.shape)
    eps = 1e-8
    fd = (m.energy(x + eps * d) - m.energy(x - eps * d)) / (2 * eps)
    assert abs(fd - np.sum(g * d)) <= 1e-6 * abs(fd)
    Hd = (m.hessian(x) @ d.ravel()).reshape(x.shape) - (m.m / m.h ** 2)[:, None] * d
    fdg = (m.grad_E(x + eps * d) - m.grad_E(x - eps * d)) / (2 * eps)
    assert np.abs(fdg - Hd).max() <= 1e-5 * np.abs(Hd).max()


def test_neohookean_pd_and_adjoint(nh_beam):
    """L-BFGS with the PD matrix A as initial Hessian reaches Newton's fixed point,
    and the adjoint matches central differences of a rollout loss in v0 and E."""
    import dataclasses
    m = TetModel(nh_beam)
    xn, _, _ = newton.newton_step(m, nh_beam.x0, nh_beam.v0, nh_beam.f_ext)
    xp, _, _ = pd_cpu.pd_lbfgs_step(m, pd_cpu.ScalarA(m), nh_beam.x0, nh_beam.v0, nh_beam.f_ext,
                                    None, None, 1e-12, 5, 5000)
    assert np.linalg.norm(xp - xn) <= 1e-9 * np.linalg.norm(xn - nh_beam.x0)
    xs, vs, _ = newton.rollout(m, nh_beam.x0, nh_beam.v0, nh_beam.f_ext, T=nh_beam.T)
    _, gx = adjoint.final_position_loss(m, xs, nh_beam.loss_w)
    g = adjoint.backward(m, xs, vs, gx)
    rng = np.random.default_rng(9)
    d = rng.standard_normal(nh_beam.x0.shape)
    d[m.dirichlet] = 0.0

    def loss(v0=None, E=None):
        mm = TetModel(nh_beam, youngs=E)
        out, _, _ = newton.rollout(mm, nh_beam.x0, nh_beam.v0 if v0 is None else v0, nh_beam.f_ext,
                                   T=nh_beam.T)
        return float(np.sum(nh_beam.loss_w * out[-1]))
    eps = 1e-6
    fd_v = (loss(v0=nh_beam.v0 + eps * d) - loss(v0=nh_beam.v0 - eps * d)) / (2 * eps)
    assert abs(fd_v - np.sum(g["g_v0"] * d)) <= 2e-6 * abs(fd_v)
    gE, _ = adjoint.material_gradients(m, g)
    dE = rng.standard_normal(m.mesh.e) * nh_beam.youngs
    fd_E = (loss(E=nh_beam.youngs + eps * dE) - loss(E=nh_beam.youngs - eps * dE)) / (2 * eps)
    assert abs(fd_E - np.sum(gE * dE)) <= 2e-6 * abs(fd_E)


@pytest.fixture(scope="module")
def ball():
    from workloads import unstructured_tet_ball
    return unstructured_tet_ball(T=8)


def test_contact_ball_derivatives_and_pd(ball):
    """Penalty ground contact on an unstructured ball (the tennis balls of Sec. 7):
    the contact term's gradient and Hessian against central differences (candidates
    kept clear of z = 0, where the penalty has its kink), and PD + L-BFGS = Newton on
    a step that starts in contact."""
    m = TetModel(ball)
    assert m.contact.sum() > 0 and m.k > 0
    rng = np.random.default_rng(10)
    x = ball.X + 0.005 * 0.01 * rng.standard_normal(ball.X.shape)
    x[:, 2] -= 0.004                                    # the lowest candidates 2 mm below ground
    zc = x[m.contact, 2]
    assert (zc < 0).sum() >= 3 and np.abs(zc).min() > 1e-5
    g = m.grad_E(x)
    d = rng.standard_normal(x.shape)
    eps = 1e-8
    fd = (m.energy(x + eps * d) - m.energy(x - eps * d)) / (2 * eps)
    assert abs(fd - np.sum(g * d)) <= 1e-6 * abs(fd)
    Hd = (m.hessian(x) @ d.ravel()).reshape(x.shape) - (m.m / m.h ** 2)[:, None] * d
    fdg = (m.grad_E(x + eps * d) - m.grad_E(x - eps * d)) / (2 * eps)
    assert np.abs(fdg - Hd).max() <= 1e-5 * np.abs(Hd).max()
    v = np.zeros_like(x)
    xn, _, _ = newton.newton_step(m, x, v, ball.f_ext)
    xp, _, _ = pd_cpu.pd_lbfgs_step(m, pd_cpu.ScalarA(m), x, v, ball.f_ext, None, None, 1e-12, 5, 5000)
    assert np.linalg.norm(xp - xn) <= 1e-8 * np.linalg.norm(xn - x)


def test_contact_ball_adjoint_matches_differences(ball):
    """The adjoint through penalty contact and Coulomb friction against central
    differences of a rollout loss in v0 and in the friction coefficient."""
    m = TetModel(ball)
    xs, vs, _ = newton.rollout(m, ball.x0, ball.v0, ball.f_ext, T=ball.T)
    assert np.any(xs[:, m.contact, 2] < 0)              # the ball reaches the ground
    _, gx = adjoint.final_position_loss(m, xs, ball.loss_w)
    g = adjoint.backward(m, xs, vs, gx)
    rng = np.random.default_rng(11)
    d = rng.standard_normal(ball.x0.shape)

    def loss(v0=None, mu=None):
        mm = TetModel(ball, mu=mu)
        out, _, _ = newton.rollout(mm, ball.x0, ball.v0 if v0 is None else v0, ball.f_ext, T=ball.T)
        return float(np.sum(ball.loss_w * out[-1]))
    eps = 1e-7
    fd_v = (loss(v0=ball.v0 + eps * d) - loss(v0=ball.v0 - eps * d)) / (2 * eps)
    assert abs(fd_v - np.sum(g["g_v0"] * d)) <= 1e-5 * abs(fd_v)
    fd_mu = (loss(mu=ball.mu + 1e-6) - loss(mu=ball.mu - 1e-6)) / 2e-6
    assert abs(fd_mu - g["g_mu"]) <= 1e-4 * max(abs(fd_mu), 1e-12)


def _complementarity_ball(T):
    import dataclasses
    from workloads import unstructured_tet_ball
    sc = unstructured_tet_ball(T=T)
    return dataclasses.replace(sc, k_contact=0.0, mu=0.0)


def test_complementarity_contact_on_the_ball():
    """Complementarity contact (Sec. 5.2, Algs 3-5; the tennis balls' ball-ground
    contact in Sec. 7) on the unstructured ball: held nodes at their targets on the
    ground, contact forces pushing, no candidate below the ground, the contact
    forces carrying the momentum change; the adjoint against central differences
    in v0 with the contact sets unchanged along the direction."""
    from oracle import contact
    sc = _complementarity_ball(4)
    model = TetModel(sc)
    cand = np.flatnonzero(sc.contact)
    xs, vs, infos = contact.rollout_complementarity(model, sc.x0, sc.v0, sc.f_ext, sc.contact, sc.T)
    assert any(i["C"].size for i in infos)
    for t, i in enumerate(infos):
        x, y = xs[t + 1], i["y"]
        assert np.array_equal(x[i["C"]], i["xstar"])
        assert np.all(i["xstar"][:, 2] == 0.0)
        assert i["rounds"] < 64
        free_set = ~np.isin(i["C"], i["locked"])
        assert np.all(i["force"][free_set, 2] >= -i["tau_r"])
        assert np.all(x[np.setdiff1d(cand, i["C"]), 2] >= -i["tau_z"])
        total = (model.m[:, None] * (x - y) / model.h ** 2).sum(axis=0)
        weight = model.m.sum() * np.linalg.norm(model.gravity)
        assert np.allclose(i["force"].sum(axis=0), total, rtol=1e-9, atol=1e-12 * weight)
    T = 3
    rng = np.random.default_rng(12)
    w = rng.standard_normal(sc.x0.shape)

    def run(v0):
        xr, vr, ir = contact.rollout_complementarity(model, sc.x0, v0, sc.f_ext, sc.contact, T)
        return float(np.sum(w * xr[-1])), xr, vr, ir
    _, xr, vr, ir = run(sc.v0)
    gx = np.zeros_like(xr)
    gx[-1] = w
    g = contact.backward_complementarity(model, xr, vr, ir, gx)
    d = rng.standard_normal(sc.v0.shape)
    eps = 1e-7
    Lp, _, _, ip = run(sc.v0 + eps * d)
    Lm, _, _, im = run(sc.v0 - eps * d)
    for a, b in zip(ip, im):
        assert np.array_equal(a["C"], b["C"]) and a["rules"] == b["rules"]
    fd = (Lp - Lm) / (2 * eps)
    an = float(np.sum(g["g_v0"] * d))
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12)
