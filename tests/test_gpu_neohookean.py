"""Neo-Hookean material on the GPU (Sec. 8) against the oracle (oracle/neohookean.py):
local step (energy and gradient) and Hessian product at small and large
deformations, FP64 and FP32; rollouts forward (L-BFGS with the PD matrix A as
initial Hessian) and backward (the splitting iteration on the Neo-Hookean Hessian)
against Newton's method and the direct adjoint, including a twisting beam with
large rotations; invalid configurations are rejected."""
import numpy as np
import pytest
import torch

from _gpu_helpers import T, make_mesh, rel
from oracle import adjoint, newton
from oracle.model import Model
from paper_2101_05917_gb300 import api
from paper_2101_05917_gb300 import _native as N
from workloads import neohookean_beam, tet_beam

pytestmark = pytest.mark.gpu

TOL = {N.PD_PREC_FP64: 1e-10, N.PD_PREC_MIXED: 2e-5}


def _state(sc, seed, scale, rotate):
    rng = np.random.default_rng(seed)
    x = sc.x0.copy()
    if rotate:
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        if np.linalg.det(Q) < 0:
            Q[:, 0] *= -1
        x = x @ Q.T
    return x + scale * sc.dx * rng.standard_normal(x.shape)


@pytest.mark.parametrize("prec", [N.PD_PREC_FP64, N.PD_PREC_MIXED])
@pytest.mark.parametrize("scale", [0.01, 0.2])   # 0.2: det F down to 0.29, no inversion
def test_local_step_and_hessian_match_oracle(prec, scale):
    sc = neohookean_beam(5, 3, 4, T=1)
    model = Model(sc)
    mesh = make_mesh(sc, precision=prec)
    rng = np.random.default_rng(2)
    for seed in range(2):
        x = _state(sc, seed, scale, rotate=seed == 1)
        g, e = mesh.local_step(T(x), precision=prec)
        assert rel(g.cpu().numpy(), model.grad_E(x)) < TOL[prec]
        e_ref = model.energy(x)
        # FP32: the energy is second order in the strain, its FP32 terms are not
        assert abs(e.item() - e_ref) <= (TOL[prec] if prec == N.PD_PREC_FP64 else 1e-3) * abs(e_ref)
        H = model.hessian(x)[model.free_dofs][:, model.free_dofs]
        v = rng.standard_normal(x.shape)
        v[model.dirichlet] = 0
        ref = np.zeros_like(v)
        ref[model.free_nodes] = (H @ v[model.free_nodes].ravel()).reshape(-1, 3)
        out = mesh.hessian_vector(T(x), T(v), precision=prec)
        assert rel(out.cpu().numpy(), ref) < TOL[prec]
    mesh.close()


@pytest.mark.parametrize("prec", [N.PD_PREC_FP64, N.PD_PREC_MIXED])
@pytest.mark.parametrize("twist", [0.0, 20.0])
def test_rollout_matches_newton_oracle(prec, twist):
    sc = neohookean_beam(5, 3, 4, T=6, twist=twist)
    model = Model(sc)
    xs, vs, _ = newton.rollout(model, sc.x0, sc.v0, sc.f_ext)
    _, gx = adjoint.final_position_loss(model, xs, sc.loss_w)
    ref = adjoint.backward(model, xs, vs, gx)
    mesh = make_mesh(sc, precision=prec)
    opts = api.solver_opts(tol_fwd=1e-10, tol_bwd=1e-10, max_iter_fwd=3000, max_iter_bwd=3000)
    f = T(sc.f_ext)
    roll = mesh.forward(T(sc.x0), T(sc.v0), sc.T, f_ext=f, opts=opts)
    g = mesh.backward(roll, sc.T, T(sc.loss_w), f_ext=f, opts=opts, want=("v0", "x0", "fext", "w_corot", "w_vol"))
    x = roll.x.cpu().numpy()
    for t in range(1, sc.T + 1):
        assert np.linalg.norm(x[t] - xs[t]) <= 1e-5 * np.linalg.norm(xs[t] - sc.x0), t
    print(f"twist {twist}: displacement-relative {np.linalg.norm(x[-1] - xs[-1]) / np.linalg.norm(xs[-1] - sc.x0):.2e}, "
          f"iterations {roll.stats['fwd_iters']} / {g['stats']['bwd_iters']}")
    for key, rkey in (("v0", "g_v0"), ("x0", "g_x0"), ("fext", "g_fext"), ("w_corot", "g_wc"), ("w_vol", "g_wv")):
        assert rel(g[key].cpu().numpy(), ref[rkey]) < 1e-4, key
    mesh.close()


def test_invalid_configurations_are_rejected():
    sc = neohookean_beam(4, 2, 3, T=1)
    dev = torch.device("cuda:0")
    mesh = api.PDMesh.from_scene(sc)
    wc, wv, _, _ = api.scene_weights(sc, dev)
    with pytest.raises(N.PDError) as err:
        mesh.factorize(wc, None, None, None, h=sc.h, neohookean=True)
    assert err.value.status == N.PD_ERR_INVALID_ARG
    mesh.close()
    st = tet_beam(T=1)
    mt = api.PDMesh.from_scene(st)
    wc, wv, _, _ = api.scene_weights(st, dev)
    with pytest.raises(N.PDError) as err:
        mt.factorize(wc, wv if wv is not None else wc, None, None, h=st.h, neohookean=True)
    assert err.value.status == N.PD_ERR_INVALID_ARG
    mt.close()
