"""Parity of unstructured tetrahedral meshes (pd_create_tet_mesh: the tetrahedral
meshes of Secs. 5.1 and 7 with their own node sets, one point per tetrahedron
with its own barycentric gradients, graph nested dissection) through the C ABI
against the FP64 oracle (oracle/tetmesh.py): local step (Eqn 20), Hessian-vector
product (Eqns 21-22), the prefactorised global solve (Eqn 19, A assembled from
the per-element gradients) and rollouts forward (Alg. 1 + L-BFGS vs Newton) and
backward (Alg. 2 + L-BFGS vs the full-linearisation adjoint), in FP64 and in the
mixed-precision path."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from _gpu_helpers import DEV, T, rel
from oracle import adjoint, newton
from oracle.tetmesh import TetModel
from paper_2101_05917_gb300 import api
from paper_2101_05917_gb300 import _native as N
from workloads import unstructured_tet_beam

pytestmark = pytest.mark.gpu

TOL = {N.PD_PREC_FP64: 1e-10, N.PD_PREC_MIXED: 2e-5}
POS_TOL = 1e-5
GRAD_TOL = 1e-4
PRECS = [N.PD_PREC_FP64, N.PD_PREC_MIXED]
SIZES = {"beam6": (6, 3, 3), "beam8": (8, 4, 4)}


def _scene(name, T_=1):
    return unstructured_tet_beam(*SIZES[name], T=T_)


def _mesh(sc, precision, leaf_max=16):
    mesh = api.PDMesh.from_tet_scene(sc, leaf_max=leaf_max, device=0)
    wc, wv, wm, fib = api.scene_weights(sc, DEV)
    mesh.factorize(wc, wv, wm, fib, h=sc.h, gravity=tuple(sc.gravity), k_contact=sc.k_contact,
                   precision=precision)
    return mesh


def _deformed(model, seed, scale=0.01, dx=0.01):
    """Rotated rest shape plus N(0, (scale dx)^2) per coordinate.  The Delaunay
    meshes keep thin tetrahedra, so the noise stays small enough that no element
    inverts (checked here): the corotated projection of an inverted element is a
    convention of its own and is not what these tests compare."""
    sc = model.scene
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    x = sc.x0 @ Q.T + scale * dx * rng.standard_normal(sc.x0.shape)
    assert np.linalg.det(model.mesh.deformation_gradients(x)[:, 0]).min() > 0.25
    return x


@pytest.mark.parametrize("name", sorted(SIZES))
@pytest.mark.parametrize("prec", PRECS)
def test_unstructured_local_step_matches_oracle(name, prec):
    sc = _scene(name)
    model = TetModel(sc)
    mesh = _mesh(sc, prec)
    for seed in range(3):
        x = _deformed(model, seed)
        g, e = mesh.local_step(T(x), None, precision=prec)
        torch.cuda.synchronize()
        assert rel(g.cpu().numpy(), model.grad_E(x)) < TOL[prec]
        e_ref = model.energy(x)
        assert abs(e.item() - e_ref) <= TOL[prec] * abs(e_ref)
    mesh.close()


@pytest.mark.parametrize("name", sorted(SIZES))
@pytest.mark.parametrize("prec", PRECS)
def test_unstructured_hessian_vector_matches_oracle(name, prec):
    sc = _scene(name)
    model = TetModel(sc)
    mesh = _mesh(sc, prec)
    rng = np.random.default_rng(7)
    x = _deformed(model, 3)
    H = model.hessian(x)[model.free_dofs][:, model.free_dofs]
    for _ in range(2):
        v = rng.standard_normal(x.shape)
        v[model.dirichlet] = 0
        ref = np.zeros_like(v)
        ref[model.free_nodes] = (H @ v[model.free_nodes].ravel()).reshape(-1, 3)
        out = mesh.hessian_vector(T(x), T(v), None, precision=prec)
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), ref) < TOL[prec]
    mesh.close()


@pytest.mark.parametrize("name", sorted(SIZES))
@pytest.mark.parametrize("leaf", [64, 8])
@pytest.mark.parametrize("prec", PRECS)
def test_unstructured_global_solve_matches_direct_solve(name, leaf, prec):
    sc = _scene(name)
    model = TetModel(sc)
    mesh = _mesh(sc, prec, leaf_max=leaf)
    A = model.A_matrix()[model.free_dofs][:, model.free_dofs].tocsc()
    rng = np.random.default_rng(1)
    b = rng.standard_normal(sc.x0.shape)
    ref = np.zeros_like(b)
    ref[model.free_nodes] = spla.spsolve(A, b[model.free_nodes].ravel()).reshape(-1, 3)
    out = mesh.solve(T(b), precision=prec)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), ref) < TOL[prec]
    mesh.close()


@pytest.mark.parametrize("prec", PRECS)
def test_unstructured_rollout_matches_oracle(prec):
    sc = _scene("beam8", T_=5)
    model = TetModel(sc)
    xs_ref, vs_ref, _ = newton.rollout(model, sc.x0, sc.v0, sc.f_ext)
    _, gx = adjoint.final_position_loss(model, xs_ref, sc.loss_w)
    ref = adjoint.backward(model, xs_ref, vs_ref, gx)
    opts = api.solver_opts(tol_fwd=1e-10, tol_bwd=1e-10, max_iter_fwd=3000, max_iter_bwd=3000)
    mesh = _mesh(sc, prec)
    f = T(sc.f_ext)
    roll = mesh.forward(T(sc.x0), T(sc.v0), sc.T, f_ext=f, opts=opts)
    g = mesh.backward(roll, sc.T, T(sc.loss_w), f_ext=f, opts=opts)
    torch.cuda.synchronize()
    xs = roll.x.cpu().numpy()
    disp = max(np.linalg.norm(xs_ref[t] - sc.x0) for t in range(1, xs_ref.shape[0]))
    err = max(np.linalg.norm(xs[t] - xs_ref[t]) for t in range(xs_ref.shape[0])) / disp
    assert err < POS_TOL
    for key, rkey in (("v0", "g_v0"), ("x0", "g_x0"), ("fext", "g_fext"), ("w_corot", "g_wc"),
                      ("w_vol", "g_wv")):
        assert rel(g[key].cpu().numpy(), ref[rkey]) < GRAD_TOL, key
    mesh.close()


def test_unstructured_rejects_muscles():
    sc = _scene("beam6")
    mesh = api.PDMesh.from_tet_scene(sc, device=0)
    wc, wv, _, _ = api.scene_weights(sc, DEV)
    e = sc.tets.shape[0]
    wm = torch.ones(e, dtype=torch.float64, device=DEV)
    fib = torch.zeros((e, 3), dtype=torch.float64, device=DEV)
    fib[:, 0] = 1.0
    with pytest.raises(N.PDError) as err:
        mesh.factorize(wc, wv, wm, fib, h=sc.h, precision=N.PD_PREC_FP64)
    assert err.value.status == N.PD_ERR_INVALID_ARG
    mesh.close()
