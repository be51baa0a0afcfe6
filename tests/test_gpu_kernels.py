"""Kernel-level parity through the C ABI: local step (Eqn 20), Hessian-vector
product (Eqns 21-22) and the prefactorised global solve (Eqn 19) against the
FP64 CPU oracle, in FP64 and in the FP32 (mixed) path."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from _gpu_helpers import DEV, T, deformed, make_mesh, rel
from oracle.model import Model
from paper_2101_05917_gb300 import _native as N
from test_oracle_dynamics import tiny_everything_scene
from workloads import cantilever_c1, quadruped, small_beam

pytestmark = pytest.mark.gpu

TOL = {N.PD_PREC_FP64: 1e-10, N.PD_PREC_MIXED: 2e-5}


def _scenes():
    return {
        "c1": cantilever_c1(T=1),
        "beam_vol": small_beam(5, 3, 4, T=1),
        "quad9": quadruped(9, T=2),
        "tiny_all": tiny_everything_scene(),
    }


@pytest.mark.parametrize("name", ["c1", "beam_vol", "quad9", "tiny_all"])
@pytest.mark.parametrize("prec", [N.PD_PREC_FP64, N.PD_PREC_MIXED])
def test_local_step_matches_oracle(name, prec):
    sc = _scenes()[name]
    model = Model(sc)
    mesh = make_mesh(sc, precision=prec)
    act = None if sc.act is None else sc.act[0]
    for seed in range(3):
        x = deformed(sc, scale=0.05, seed=seed)
        if sc.k_contact > 0:
            x[:, 2] -= 0.3 * sc.dx   # put some contact candidates below the ground
        g_ref = model.grad_E(x, act)
        e_ref = model.energy(x, act)
        g, e = mesh.local_step(T(x), None if act is None else T(act), precision=prec)
        torch.cuda.synchronize()
        assert rel(g.cpu().numpy(), g_ref) < TOL[prec]
        assert abs(e.item() - e_ref) <= TOL[prec] * abs(e_ref)
    mesh.close()


@pytest.mark.parametrize("name", ["c1", "beam_vol", "quad9", "tiny_all"])
@pytest.mark.parametrize("prec", [N.PD_PREC_FP64, N.PD_PREC_MIXED])
def test_hessian_vector_matches_oracle(name, prec):
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


@pytest.mark.parametrize("name", ["c1", "beam_vol", "quad9", "tiny_all"])
@pytest.mark.parametrize("leaf", [64, 8])
@pytest.mark.parametrize("prec", [N.PD_PREC_FP64, N.PD_PREC_MIXED])
def test_global_solve_matches_direct_solve(name, leaf, prec):
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


@pytest.mark.parametrize("name", ["c1", "beam_vol", "quad9"])
def test_strain_accurate_local_step_under_large_rotation(name):
    """A random rigid rotation with a strain of ~1e-4 on top: H = F - I is of the
    order of the rotation while the stresses are of the order of the strain.  The
    strain-accurate FP32 local step (F - I and the Green strain in FP64) matches the
    oracle's gradient and Hessian product within the FP32 tolerance; the plain FP32
    step's error is printed beside it (it grows with rotation / strain)."""
    sc = _scenes()[name]
    model = Model(sc)
    mesh = make_mesh(sc, precision=N.PD_PREC_MIXED)
    act = None if sc.act is None else sc.act[0]
    x = deformed(sc, scale=1e-4, seed=11)
    g_ref = model.grad_E(x, act)
    e_ref = model.energy(x, act)
    ta = None if act is None else T(act)
    g_acc, e_acc = mesh.local_step(T(x), ta, precision=N.PD_PREC_MIXED_STRAIN)
    g_32, _ = mesh.local_step(T(x), ta, precision=N.PD_PREC_MIXED)
    torch.cuda.synchronize()
    err_acc, err_32 = rel(g_acc.cpu().numpy(), g_ref), rel(g_32.cpu().numpy(), g_ref)
    print(f"{name}: strain-accurate {err_acc:.2e}, plain FP32 {err_32:.2e}")
    assert err_acc < TOL[N.PD_PREC_MIXED]
    assert abs(e_acc.item() - e_ref) <= TOL[N.PD_PREC_MIXED] * abs(e_ref)
    H = model.hessian(x, act)[model.free_dofs][:, model.free_dofs]
    v = np.random.default_rng(3).standard_normal(x.shape)
    v[model.dirichlet] = 0
    ref = np.zeros_like(v)
    ref[model.free_nodes] = (H @ v[model.free_nodes].ravel()).reshape(-1, 3)
    out = mesh.hessian_vector(T(x), T(v), ta, precision=N.PD_PREC_MIXED_STRAIN)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), ref) < TOL[N.PD_PREC_MIXED]
    mesh.close()


def _quad9_corot_muscle():
    sc = quadruped(9, T=2)
    sc.volume = False          # corotated + muscle + contact: the refined kernel's energies
    return sc


@pytest.mark.parametrize("name", ["c1", "quad9_corot_muscle", "quad9", "tiny_all"])
@pytest.mark.parametrize("scale", [0.05, 1e-4])
def test_refined_fp64_local_step_matches_oracle(name, scale):
    """PD_PREC_FP64_REFINED (FP32 SVD of the FP64 strain, rotation and its
    derivative refined in FP64 without eigenvectors) gives the gradient and the
    Hessian product to FP64 accuracy: against the oracle within the FP64 tolerance
    and against the plain FP64 kernel within 1e-12, at moderate strain (0.05) and
    at a strain of 1e-4 under a random rotation.  Meshes with the volume energy run
    the plain FP64 kernel through the same entry (checked for equality).  At a
    strain of 1e-4 the gradient is 1e4 times smaller than the positions it comes
    from, so two FP64 evaluations agree to ~1e-11 there: the gate is 1e-9."""
    sc = _quad9_corot_muscle() if name == "quad9_corot_muscle" else _scenes()[name]
    model = Model(sc)
    mesh = make_mesh(sc, precision=N.PD_PREC_MIXED)
    act = None if sc.act is None else sc.act[0]
    ta = None if act is None else T(act)
    x = deformed(sc, scale=scale, seed=13)
    if sc.k_contact > 0:
        x[:, 2] -= 0.3 * sc.dx
    g_ref = model.grad_E(x, act)
    g_r, e_r = mesh.local_step(T(x), ta, precision=N.PD_PREC_FP64_REFINED)
    g_d, e_d = mesh.local_step(T(x), ta, precision=N.PD_PREC_FP64)
    torch.cuda.synchronize()
    gr, gd = g_r.cpu().numpy(), g_d.cpu().numpy()
    tol = TOL[N.PD_PREC_FP64] if scale > 1e-3 else 1e-9
    print(f"{name} strain {scale}: refined vs oracle {rel(gr, g_ref):.2e}, vs FP64 kernel {rel(gr, gd):.2e}")
    assert rel(gr, g_ref) < tol
    assert rel(gr, gd) < tol
    assert abs(e_r.item() - e_d.item()) <= tol * abs(e_d.item())
    H = model.hessian(x, act)[model.free_dofs][:, model.free_dofs]
    v = np.random.default_rng(4).standard_normal(x.shape)
    v[model.dirichlet] = 0
    ref = np.zeros_like(v)
    ref[model.free_nodes] = (H @ v[model.free_nodes].ravel()).reshape(-1, 3)
    h_r = mesh.hessian_vector(T(x), T(v), ta, precision=N.PD_PREC_FP64_REFINED).cpu().numpy()
    h_d = mesh.hessian_vector(T(x), T(v), ta, precision=N.PD_PREC_FP64).cpu().numpy()
    assert rel(h_r, ref) < tol
    assert rel(h_r, h_d) < tol
    mesh.close()
