"""Parity of the tetrahedral element rule (six linear tetrahedra per voxel cell,
one point each; stands in for the tetrahedral meshes of Secs. 5.1 and 7)
through the C ABI against the FP64 oracle: local step (Eqn 20), Hessian-vector
product (Eqns 21-22), the prefactorised global solve (Eqn 19, A assembled from
the tetrahedra) and rollouts forward (Alg. 1 + L-BFGS vs Newton) and backward
(Alg. 2 + L-BFGS vs the full-linearisation adjoint), with contact, friction and
muscles, in FP64 and in the mixed-precision path."""
import dataclasses

import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from _gpu_helpers import T, deformed, make_mesh, rel
from oracle import adjoint, newton
from oracle.model import Model
from paper_2101_05917_gb300 import api
from paper_2101_05917_gb300 import _native as N
from test_oracle_dynamics import tiny_everything_scene
from workloads import tet_ball, tet_beam

pytestmark = pytest.mark.gpu

TOL = {N.PD_PREC_FP64: 1e-10, N.PD_PREC_MIXED: 2e-5}
POS_TOL = 1e-5
GRAD_TOL = 1e-4


def _tet_all(T_=3):
    return dataclasses.replace(tiny_everything_scene(T=T_), element_rule="tet6", name="tiny_tet")


def _scenes():
    return {"tet_beam": tet_beam(5, 3, 4, T=1), "tet_all": _tet_all(), "tet_ball": tet_ball(T=1)}


NAMES = ["tet_beam", "tet_all", "tet_ball"]
PRECS = [N.PD_PREC_FP64, N.PD_PREC_MIXED]


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", PRECS)
def test_tet_local_step_matches_oracle(name, prec):
    sc = _scenes()[name]
    model = Model(sc)
    mesh = make_mesh(sc, precision=prec)
    act = None if sc.act is None else sc.act[0]
    for seed in range(3):
        x = deformed(sc, scale=0.05, seed=seed)
        if sc.k_contact > 0:
            x[:, 2] -= 0.3 * sc.dx
        g_ref = model.grad_E(x, act)
        e_ref = model.energy(x, act)
        g, e = mesh.local_step(T(x), None if act is None else T(act), precision=prec)
        torch.cuda.synchronize()
        assert rel(g.cpu().numpy(), g_ref) < TOL[prec]
        assert abs(e.item() - e_ref) <= TOL[prec] * abs(e_ref)
    mesh.close()


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("prec", PRECS)
def test_tet_hessian_vector_matches_oracle(name, prec):
    sc = _scenes()[name]
    model = Model(sc)
    mesh = make_mesh(sc, precision=prec)
    act = None if sc.act is None else sc.act[0]
    rng = np.random.default_rng(7)
    x = deformed(sc, scale=0.05, seed=3)
    if sc.k_contact > 0:
        x[:, 2] -= 0.3 * sc.dx
    H = model.hessian(x, act)[model.free_dofs][:, model.free_dofs]
    for _ in range(2):
        v = rng.standard_normal(x.shape)
        v[model.dirichlet] = 0
        ref = np.zeros_like(v)
        ref[model.free_nodes] = (H @ v[model.free_nodes].ravel()).reshape(-1, 3)
        out = mesh.hessian_vector(T(x), T(v), None if act is None else T(act), precision=prec)
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), ref) < TOL[prec]
    mesh.close()


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("leaf", [64, 8])
@pytest.mark.parametrize("prec", PRECS)
def test_tet_global_solve_matches_direct_solve(name, leaf, prec):
    sc = _scenes()[name]
    model = Model(sc)
    mesh = make_mesh(sc, precision=prec, leaf_max=leaf)
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
@pytest.mark.parametrize("name", NAMES)
def test_tet_rollout_matches_oracle(name, prec):
    sc = {"tet_beam": tet_beam(5, 3, 4, T=6), "tet_all": _tet_all(4), "tet_ball": tet_ball(T=10)}[name]
    model = Model(sc)
    xs_ref, vs_ref, _ = newton.rollout(model, sc.x0, sc.v0, sc.f_ext, sc.act)
    if sc.k_contact > 0:
        assert np.any(xs_ref[:, model.contact, 2] < 0)
    _, gx = adjoint.final_position_loss(model, xs_ref, sc.loss_w)
    ref = adjoint.backward(model, xs_ref, vs_ref, gx, act=sc.act)
    opts = api.solver_opts(tol_fwd=1e-10, tol_bwd=1e-10, max_iter_fwd=3000, max_iter_bwd=3000)
    mesh = make_mesh(sc, precision=prec)
    f = T(sc.f_ext)
    act = None if sc.act is None else T(sc.act)
    roll = mesh.forward(T(sc.x0), T(sc.v0), sc.T, f_ext=f, act=act, mu=sc.mu, opts=opts)
    g = mesh.backward(roll, sc.T, T(sc.loss_w), f_ext=f, act=act, mu=sc.mu, opts=opts)
    torch.cuda.synchronize()
    xs = roll.x.cpu().numpy()
    err = max(np.linalg.norm(xs[t] - xs_ref[t]) / np.linalg.norm(xs_ref[t]) for t in range(xs_ref.shape[0]))
    assert err < POS_TOL
    for key, rkey in (("v0", "g_v0"), ("x0", "g_x0"), ("fext", "g_fext"), ("w_corot", "g_wc"),
                      ("w_vol", "g_wv")):
        assert rel(g[key].cpu().numpy(), ref[rkey]) < GRAD_TOL, key
    if sc.act is not None:
        assert rel(g["act"].cpu().numpy(), ref["g_act"]) < GRAD_TOL
        assert rel(g["w_muscle"].cpu().numpy(), ref["g_wm"]) < GRAD_TOL
    if sc.k_contact > 0 and sc.mu > 0:
        assert abs(g["mu"].item() - ref["g_mu"]) <= GRAD_TOL * max(abs(ref["g_mu"]), 1e-12)
    mesh.close()
