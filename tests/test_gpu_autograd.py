"""torch.autograd over the rollout: gradients of a loss on every state (positions
and velocities) w.r.t. x0, v0, f_ext, actuation, material weights and mu match
central finite differences of the same loss (FP64 path, tight tolerances)."""
import numpy as np
import pytest
import torch

from paper_2101_05917_gb300 import _native as N
from paper_2101_05917_gb300 import api
from paper_2101_05917_gb300.autograd import Simulator
from workloads import quadruped, small_beam

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
# the quadruped (contact, random 30 % muscle contraction) converges slowly: a looser
# solve tolerance (1e-11) with a larger finite-difference step keeps the FD noise below
# the gate (at 1e-10 the loss noise, ~1e-8, is already ~1e-4 of the central difference)
CASES = {"beam": dict(opts=dict(tol_fwd=1e-12, tol_bwd=1e-12, max_iter_fwd=5000, max_iter_bwd=5000),
                      eps=1e-6, rtol=2e-5),
         "quadruped": dict(opts=dict(tol_fwd=1e-11, tol_bwd=1e-11, max_iter_fwd=50000, max_iter_bwd=50000),
                           eps=1e-4, rtol=1e-4,
                           # absolute steps: large enough that the loss noise left by the
                           # 1e-11 solves (~1e-9) stays far below the gate
                           abs_eps={"v0": 1e-4, "f_ext": 1e-4, "act": 1e-4, "mu": 1e-4})}


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _inputs(sc, T):
    wc, wv, wm, fib = api.scene_weights(sc, DEV)
    d = {"x0": _t(sc.x0), "v0": _t(sc.v0), "f_ext": _t(sc.f_ext), "w_corot": wc, "w_vol": wv}
    if wm is not None:
        d["w_muscle"] = wm
        d["act"] = _t(sc.act[:T])
    d["mu"] = torch.tensor(float(sc.mu), dtype=torch.float64, device=DEV)
    return d, fib


def _loss(sim, d, fib, T, cx, cv):
    x, v = sim.rollout(d["x0"], d["v0"], T, f_ext=d["f_ext"], act=d.get("act"), w_corot=d["w_corot"],
                       w_vol=d["w_vol"], w_muscle=d.get("w_muscle"), fiber=fib, mu=d["mu"])
    return (x * cx).sum() + (v[-1] * cv).sum()


@pytest.mark.parametrize("which", ["beam", "quadruped"])
def test_autograd_matches_finite_differences(which):
    T = 3
    sc = small_beam(4, 2, 2, T=T) if which == "beam" else quadruped(4, T=T)
    case = CASES[which]
    sim = Simulator.from_scene(sc, precision=N.PD_PREC_FP64, opts=case["opts"])
    d, fib = _inputs(sc, T)
    rng = np.random.default_rng(11)
    n = sc.x0.shape[0]
    cx = _t(rng.standard_normal((T + 1, n, 3)))
    cv = _t(rng.standard_normal((n, 3)))
    leaves = {k: v.clone().requires_grad_(True) for k, v in d.items()}
    loss = _loss(sim, leaves, fib, T, cx, cv)
    loss.backward()
    # the quadruped's feet start exactly on the ground (z = 0), where friction
    # switches on for z < 0: a finite difference in x0 would cross that branch
    names = ["x0", "v0", "f_ext", "w_corot", "w_vol"] if which == "beam" else \
        ["v0", "f_ext", "w_corot", "w_vol", "w_muscle", "act", "mu"]
    for name in names:
        g = leaves[name].grad
        assert g is not None, name
        base = d[name]
        direc = _t(rng.standard_normal(tuple(base.shape)))
        if name == "act":
            direc = direc * (base > 0)        # leg elements only
        scale = float(base.abs().max()) if name not in ("x0",) else 1.0
        eps = case.get("abs_eps", {}).get(name, case["eps"] * max(scale, 1e-3))
        dp = dict(d)
        dm = dict(d)
        dp[name] = base + eps * direc
        dm[name] = base - eps * direc
        with torch.no_grad():
            fd = (float(_loss(sim, dp, fib, T, cx, cv)) - float(_loss(sim, dm, fib, T, cx, cv))) / (2 * eps)
        an = float((g * direc).sum())
        assert abs(fd - an) <= case["rtol"] * max(abs(an), 1e-8) + 1e-9, (name, fd, an)
    sim.mesh.close()


def test_autograd_with_checkpoints_equals_stored_states():
    """With checkpoint_every = K the wrapper returns the checkpointed states only;
    a loss on them back-propagates (states recomputed per segment, Sec. 4) to
    gradients bit-identical to those of the same loss on the stored trajectory."""
    T, K = 4, 2
    sc = small_beam(4, 2, 2, T=T)
    opts = dict(tol_fwd=1e-11, tol_bwd=1e-11, max_iter_fwd=5000, max_iter_bwd=5000)
    d, fib = _inputs(sc, T)
    rng = np.random.default_rng(12)
    n = sc.x0.shape[0]
    cx = _t(rng.standard_normal((T // K + 1, n, 3)))
    cv = _t(rng.standard_normal((T // K + 1, n, 3)))
    grads = []
    for every in (0, K):
        sim = Simulator.from_scene(sc, precision=N.PD_PREC_FP64, opts=dict(opts, checkpoint_every=every))
        leaves = {k: v.clone().requires_grad_(True) for k, v in d.items()}
        x, v = sim.rollout(leaves["x0"], leaves["v0"], T, f_ext=leaves["f_ext"], w_corot=leaves["w_corot"],
                           w_vol=leaves["w_vol"], mu=leaves["mu"])
        if every == 0:
            x, v = x[::K], v[::K]
        assert x.shape == (T // K + 1, n, 3)
        ((x * cx).sum() + (v * cv).sum()).backward()
        grads.append({k: leaves[k].grad.clone() for k in ("x0", "v0", "f_ext", "w_corot", "w_vol")})
        sim.mesh.close()
    for k in grads[0]:
        assert torch.equal(grads[0][k], grads[1][k]), k
