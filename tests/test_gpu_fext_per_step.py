"""External force given per step (f_ext of shape (T, n, 3), pd_solver_opts
fext_per_step): step t's predictor uses slice t (Sec. 3, Eqn 1) and the backward
pass returns dL/df_ext[t] = z_t, the adjoint of step t (Eqns 8-12: y depends on
f_ext through h^2 M^-1 and dL/dy = M z / h^2).

Checks: a per-step force equal in every step reproduces the constant-force run bit
for bit, and its per-step gradients add up (in the library's order) to the summed
gradient exactly; a force that varies per step matches the Newton oracle stepped
with the same slices and the oracle adjoint's per-step z_t (1e-5 / 1e-4, FP64 and
mixed precision), with checkpointing as well; wrong shapes are rejected."""
import numpy as np
import pytest
import torch

from _gpu_helpers import T, make_mesh, rel
from oracle import adjoint, newton
from oracle.model import Model
from paper_2101_05917_gb300 import api
from paper_2101_05917_gb300 import _native as N
from workloads import small_beam

pytestmark = pytest.mark.gpu


def _forces(sc, steps, seed):
    """Per-step external force: the scene's traction scaled per step plus a seeded
    random field on the free nodes (same order of magnitude)."""
    rng = np.random.default_rng(seed)
    scale = 1.0 + 0.5 * rng.standard_normal(steps)
    mag = np.abs(sc.f_ext).max() if np.abs(sc.f_ext).max() > 0 else 1e-4
    f = sc.f_ext[None] * scale[:, None, None] + 0.3 * mag * rng.standard_normal((steps,) + sc.f_ext.shape)
    f[:, sc.dirichlet > 0] = 0.0
    return f


@pytest.mark.parametrize("prec", [N.PD_PREC_FP64, N.PD_PREC_MIXED])
def test_constant_slices_reproduce_constant_force(prec):
    sc = small_beam(5, 3, 4, T=6)
    mesh = make_mesh(sc, precision=prec)
    opts = api.solver_opts(tol_fwd=1e-10, tol_bwd=1e-10, max_iter_fwd=3000, max_iter_bwd=3000)
    f = T(sc.f_ext)
    fs = T(np.repeat(sc.f_ext[None], sc.T, axis=0))
    lw = T(sc.loss_w)
    r1 = mesh.forward(T(sc.x0), T(sc.v0), sc.T, f_ext=f, opts=opts)
    g1 = mesh.backward(r1, sc.T, lw, f_ext=f, opts=opts, want=("v0", "fext"))
    r2 = mesh.forward(T(sc.x0), T(sc.v0), sc.T, f_ext=fs, opts=opts)
    g2 = mesh.backward(r2, sc.T, lw, f_ext=fs, opts=opts, want=("v0", "fext"))
    assert torch.equal(r1.x, r2.x) and torch.equal(r1.v, r2.v)
    assert torch.equal(g1["v0"], g2["v0"])
    assert tuple(g2["fext"].shape) == (sc.T, sc.x0.shape[0], 3)
    acc = torch.zeros_like(g1["fext"])
    for t in reversed(range(sc.T)):   # the order in which the summed gradient accumulates
        acc += g2["fext"][t]
    assert torch.equal(acc, g1["fext"])
    mesh.close()


@pytest.mark.parametrize("prec,K", [(N.PD_PREC_FP64, 0), (N.PD_PREC_MIXED, 0), (N.PD_PREC_MIXED, 3)])
def test_varying_force_matches_oracle(prec, K):
    sc = small_beam(5, 3, 4, T=6)
    fs = _forces(sc, sc.T, seed=11)
    model = Model(sc)
    xs = [sc.x0.copy()]
    vs = [sc.v0.copy()]
    for t in range(sc.T):
        xn, vn, _ = newton.newton_step(model, xs[-1], vs[-1], fs[t])
        xs.append(xn)
        vs.append(vn)
    xs, vs = np.stack(xs), np.stack(vs)
    _, gx = adjoint.final_position_loss(model, xs, sc.loss_w)
    ref = adjoint.backward(model, xs, vs, gx)
    mesh = make_mesh(sc, precision=prec)
    opts = api.solver_opts(tol_fwd=1e-10, tol_bwd=1e-10, max_iter_fwd=3000, max_iter_bwd=3000,
                           checkpoint_every=K)
    f = T(fs)
    roll = mesh.forward(T(sc.x0), T(sc.v0), sc.T, f_ext=f, opts=opts)
    g = mesh.backward(roll, sc.T, T(sc.loss_w), f_ext=f, opts=opts, want=("v0", "fext"))
    x_last = roll.x[-1].cpu().numpy()
    assert rel(x_last, xs[-1]) < 1e-5
    assert np.linalg.norm(x_last - xs[-1]) / np.linalg.norm(xs[-1] - sc.x0) < 1e-5
    gf = g["fext"].cpu().numpy()
    tol = 1e-7 if prec == N.PD_PREC_FP64 else 1e-4
    for t in range(sc.T):
        assert rel(gf[t], ref["zs"][t]) < tol, t
    assert rel(g["v0"].cpu().numpy(), ref["g_v0"]) < tol
    mesh.close()


def test_wrong_force_shape_is_rejected():
    sc = small_beam(4, 2, 2, T=3)
    mesh = make_mesh(sc)
    bad = T(np.zeros((sc.T + 1,) + sc.x0.shape))
    with pytest.raises(ValueError):
        mesh.forward(T(sc.x0), T(sc.v0), sc.T, f_ext=bad)
    mesh.close()
