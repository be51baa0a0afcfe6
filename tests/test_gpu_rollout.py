"""Rollout parity through the C ABI: PD forward (Alg. 1 + L-BFGS) against the
Newton oracle (Sec. 3) and the PD adjoint (Alg. 2 + L-BFGS) against the
full-linearisation adjoint (Eqns 8-12).  Gates: 1e-5 relative position error
(max over steps), the same relative to the displacement |x_t - X| and, per
component, relative to the largest displacement component; 1e-4 relative
gradient error."""
import os

import numpy as np
import pytest
import torch

from _gpu_helpers import DEV, T, make_mesh, rel
from oracle import adjoint, newton
from oracle.model import Model
from paper_2101_05917_gb300 import api
from paper_2101_05917_gb300 import _native as N
from test_oracle_dynamics import tiny_everything_scene
from workloads import cantilever_c1, quadruped, small_beam

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "c1_cantilever_oracle.npz")
POS_TOL = 1e-5
GRAD_TOL = 1e-4


def _pos_err(xs, ref):
    return max(np.linalg.norm(xs[t] - ref[t]) / np.linalg.norm(ref[t]) for t in range(ref.shape[0]))


def _disp_errs(xs, ref):
    """(|dx| / |x_t - X|, max|dx| / max|x_t - X|), worst over steps t >= 1."""
    X = ref[0]
    d = max(np.linalg.norm(xs[t] - ref[t]) / np.linalg.norm(ref[t] - X) for t in range(1, ref.shape[0]))
    m = max(np.abs(xs[t] - ref[t]).max() / np.abs(ref[t] - X).max() for t in range(1, ref.shape[0]))
    return float(d), float(m)


def _run(sc, prec, opts, loss_all_steps=False):
    mesh = make_mesh(sc, precision=prec)
    f = T(sc.f_ext)
    act = None if sc.act is None else T(sc.act)
    roll = mesh.forward(T(sc.x0), T(sc.v0), sc.T, f_ext=f, act=act, mu=sc.mu, opts=opts)
    g = mesh.backward(roll, sc.T, T(sc.loss_w), f_ext=f, act=act, mu=sc.mu, opts=opts)
    torch.cuda.synchronize()
    return mesh, roll, g


def test_c1_cantilever_fp64_matches_oracle():
    sc = cantilever_c1()
    gold = np.load(GOLD)
    opts = api.solver_opts(tol_fwd=1e-9, tol_bwd=1e-9)
    mesh, roll, g = _run(sc, N.PD_PREC_FP64, opts)
    xs = roll.x.cpu().numpy()
    assert _pos_err(xs, gold["xs"]) < POS_TOL
    assert np.abs(xs - gold["xs"]).max() < 1e-8
    d, m = _disp_errs(xs, gold["xs"])
    print(f"C1 displacement-relative {d:.2e}, component max {m:.2e}")
    assert d < POS_TOL and m < POS_TOL
    assert rel(g["v0"].cpu().numpy(), gold["g_v0"]) < GRAD_TOL
    assert rel(g["x0"].cpu().numpy(), gold["g_x0"]) < GRAD_TOL
    assert rel(g["w_corot"].cpu().numpy(), gold["g_wc"]) < GRAD_TOL
    # dL/dE and dL/dnu through w_corot = E/(1+nu)
    nu = sc.poisson
    gE = g["w_corot"].cpu().numpy() / (1 + nu)
    gnu = float(np.sum(g["w_corot"].cpu().numpy() * (-sc.youngs / (1 + nu) ** 2)))
    assert rel(gE, gold["g_E"]) < GRAD_TOL
    assert abs(gnu - float(gold["g_nu"])) < GRAD_TOL * abs(float(gold["g_nu"]))
    st = roll.stats
    assert st["not_converged_steps"] == 0 and st["max_fwd_rel_residual"] <= 1e-9
    mesh.close()


@pytest.mark.parametrize("prec", [N.PD_PREC_FP64, N.PD_PREC_MIXED])
@pytest.mark.parametrize("name", ["beam_vol", "tiny_all", "quad8"])
def test_rollout_matches_oracle(name, prec):
    sc = {"beam_vol": small_beam(5, 3, 4, T=6), "tiny_all": tiny_everything_scene(T=4),
          "quad8": quadruped(8, T=4)}[name]
    model = Model(sc)
    xs_ref, vs_ref, _ = newton.rollout(model, sc.x0, sc.v0, sc.f_ext, sc.act)
    _, gx = adjoint.final_position_loss(model, xs_ref, sc.loss_w)
    ref = adjoint.backward(model, xs_ref, vs_ref, gx, act=sc.act)
    # free-floating bodies on the ground converge slowly (near-rigid rotations)
    opts = api.solver_opts(tol_fwd=1e-10, tol_bwd=1e-10, max_iter_fwd=3000, max_iter_bwd=3000)
    mesh, roll, g = _run(sc, prec, opts)
    xs = roll.x.cpu().numpy()
    assert _pos_err(xs, xs_ref) < POS_TOL
    d, m = _disp_errs(xs, xs_ref)
    print(f"{name}: displacement-relative {d:.2e}, component max {m:.2e}")
    assert d < POS_TOL and m < POS_TOL
    for key, rkey in (("v0", "g_v0"), ("x0", "g_x0"), ("fext", "g_fext")):
        assert rel(g[key].cpu().numpy(), ref[rkey]) < GRAD_TOL, key
    if sc.corotated:
        assert rel(g["w_corot"].cpu().numpy(), ref["g_wc"]) < GRAD_TOL
    if sc.volume:
        assert rel(g["w_vol"].cpu().numpy(), ref["g_wv"]) < GRAD_TOL
    if sc.act is not None:
        assert rel(g["act"].cpu().numpy(), ref["g_act"]) < GRAD_TOL
        assert rel(g["w_muscle"].cpu().numpy(), ref["g_wm"]) < GRAD_TOL
    if sc.k_contact > 0 and sc.mu > 0:
        assert abs(g["mu"].item() - ref["g_mu"]) <= GRAD_TOL * max(abs(ref["g_mu"]), 1e-12)
    mesh.close()


@pytest.mark.parametrize("prec", [N.PD_PREC_FP64, N.PD_PREC_MIXED])
def test_checkpointed_backward_is_bit_identical(prec):
    """Mixed precision at tol 1e-10 sits below the FP32 floor: the forward steps
    switch to the strain-accurate tier, which stays on for later steps and across
    the checkpoint at step 4; the recomputation replays the forward's tier state."""
    sc = small_beam(4, 3, 3, T=8)
    opts = api.solver_opts(tol_fwd=1e-10, tol_bwd=1e-10)
    mesh = make_mesh(sc, precision=prec)
    f = T(sc.f_ext)
    roll = mesh.forward(T(sc.x0), T(sc.v0), sc.T, f_ext=f, opts=opts)
    g_full = mesh.backward(roll, sc.T, T(sc.loss_w), f_ext=f, opts=opts)
    opts_ck = api.solver_opts(tol_fwd=1e-10, tol_bwd=1e-10, checkpoint_every=4)
    roll_ck = mesh.forward(T(sc.x0), T(sc.v0), sc.T, f_ext=f, opts=opts_ck)
    assert torch.equal(roll_ck.x[1], roll.x[4]) and torch.equal(roll_ck.x[2], roll.x[8])
    g_ck = mesh.backward(roll_ck, sc.T, T(sc.loss_w), f_ext=f, opts=opts_ck)
    for k in ("x0", "v0", "fext", "w_corot", "w_vol"):
        assert torch.equal(g_full[k], g_ck[k]), k
    mesh.close()


def test_runs_are_deterministic():
    sc = small_beam(5, 3, 4, T=4)
    opts = api.solver_opts(tol_fwd=1e-10, tol_bwd=1e-10)
    outs = []
    for _ in range(2):
        mesh, roll, g = _run(sc, N.PD_PREC_MIXED, opts)
        outs.append((roll.x.clone(), g["v0"].clone(), g["w_vol"].clone()))
        mesh.close()
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)


def test_checkpointing_planned_from_a_memory_cap_is_bit_identical():
    """A memory cap too small for all T+1 states makes the forward pass checkpoint
    on its own (pd_plan_checkpoints picks the interval); the backward pass then
    recomputes each segment and the gradients equal those over stored states bit
    for bit (Sec. 4, back-propagation through every step)."""
    steps = 8
    sc = small_beam(4, 2, 2, T=steps)
    mesh = make_mesh(sc)
    state = 48 * mesh.n
    want = ("x0", "v0", "fext", "w_corot", "w_vol")
    outs = []
    for every, cap in ((0, 0), (-1, 8 * state)):
        o = api.solver_opts(tol_fwd=1e-11, tol_bwd=1e-11, max_iter_fwd=5000, max_iter_bwd=5000,
                            checkpoint_every=every)
        roll = mesh.forward(T(sc.x0), T(sc.v0), steps, f_ext=T(sc.f_ext), opts=o, mem_cap=cap)
        g = mesh.backward(roll, steps, T(sc.loss_w), f_ext=T(sc.f_ext), opts=o, want=want)
        outs.append((roll, g))
    assert outs[0][0].checkpoint_every == 0 and outs[1][0].checkpoint_every == 2
    assert torch.equal(outs[0][0].x[-1], outs[1][0].x[-1])
    for k in want:
        assert torch.equal(outs[0][1][k], outs[1][1][k]), k
    mesh.close()
