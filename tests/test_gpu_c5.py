"""Large cantilever (64x64x128 cells, 1,635,075 DoFs, surface tractions), first 4
steps with checkpoints every 2 steps (Sec. 4: states recomputed per segment in the
backward pass).  No CPU oracle finishes at this size, so the checks are: the
checkpointed backward pass is bit-identical to the one over stored states, mixed
precision agrees with FP64, and the FP64 gradient w.r.t. the traction field matches
central finite differences of the loss along seeded unit directions."""
import numpy as np
import pytest
import torch

from paper_2101_05917_gb300 import _native as N
from paper_2101_05917_gb300 import api
from workloads import beam_c5

pytestmark = pytest.mark.gpu

T = 4
DEV = torch.device("cuda:0")


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def c5():
    sc = beam_c5(T=T)
    mesh = api.PDMesh.from_scene(sc)
    wc, wv, _, _ = api.scene_weights(sc, DEV)
    yield sc, mesh, wc, wv
    mesh.close()


def _factor(c5, precision):
    sc, mesh, wc, wv = c5
    mesh.factorize(wc, wv, None, None, h=sc.h, gravity=tuple(sc.gravity), precision=precision)


def _rollout(c5, tol, K, f_ext=None, backward=True):
    sc, mesh, _, _ = c5
    f = _t(sc.f_ext) if f_ext is None else f_ext
    opts = api.solver_opts(tol_fwd=tol, tol_bwd=tol, max_iter_fwd=5000, max_iter_bwd=5000, checkpoint_every=K)
    roll = mesh.forward(_t(sc.x0), _t(sc.v0), T, f_ext=f, opts=opts)
    if not backward:
        return roll, None
    g = mesh.backward(roll, T, _t(sc.loss_w), f_ext=f, opts=opts, want=("v0", "fext"))
    return roll, g


def test_c5_checkpoints_mixed_vs_fp64_and_fd(c5):
    sc = c5[0]
    _factor(c5, N.PD_PREC_MIXED)
    r_k, g_k = _rollout(c5, 1e-7, 2)
    r_f, g_f = _rollout(c5, 1e-7, 0)
    # checkpointed states are the stored ones; recomputation is bit-identical
    assert torch.equal(r_k.x[-1], r_f.x[-1])
    assert torch.equal(g_k["fext"], g_f["fext"]) and torch.equal(g_k["v0"], g_f["v0"])
    _factor(c5, N.PD_PREC_FP64)
    r_d, g_d = _rollout(c5, 1e-10, 2)
    x_mixed, x_fp64 = r_k.x[-1].cpu().numpy(), r_d.x[-1].cpu().numpy()
    pos = np.linalg.norm(x_mixed - x_fp64) / np.linalg.norm(x_fp64)
    gm, gd = g_k["fext"].cpu().numpy(), g_d["fext"].cpu().numpy()
    grad = np.linalg.norm(gm - gd) / np.linalg.norm(gd)
    gv = np.linalg.norm(g_k["v0"].cpu().numpy() - g_d["v0"].cpu().numpy()) / np.linalg.norm(g_d["v0"].cpu().numpy())
    print(f"C5 mixed vs FP64: position {pos:.2e}, grad f_ext {grad:.2e}, grad v0 {gv:.2e}")
    assert pos <= 1e-5 and grad <= 1e-4 and gv <= 1e-4
    # central differences along seeded unit directions of the traction field (FP64)
    rng = np.random.default_rng(5025)
    surf = np.abs(sc.f_ext).sum(axis=1) > 0
    lw = _t(sc.loss_w)
    for k in range(2):
        d = np.zeros_like(sc.f_ext)
        d[surf] = rng.standard_normal((int(surf.sum()), 3))
        d /= np.linalg.norm(d)
        eps = 1e-3
        lp = float((_rollout(c5, 1e-10, 2, f_ext=_t(sc.f_ext + eps * d), backward=False)[0].x[-1] * lw).sum())
        lm = float((_rollout(c5, 1e-10, 2, f_ext=_t(sc.f_ext - eps * d), backward=False)[0].x[-1] * lw).sum())
        fd = (lp - lm) / (2 * eps)
        an = float(np.sum(gd * d))
        print(f"C5 FD direction {k}: fd {fd:.10e} adjoint {an:.10e}")
        assert abs(fd - an) <= 1e-4 * abs(an)


def test_c5_benchmark_configuration_matches_fp64_over_50_steps(c5):
    """The configuration bench.py times (mixed precision, tol 1e-7, checkpoints every
    25 steps) over the first 50 steps against the FP64 path at tol 1e-10 (the FP64
    path is pinned to the oracle on the small meshes; no CPU oracle finishes at this
    size).  Gates: relative position error 1e-5, displacement-relative error and
    element-wise maximum (scaled by the largest displacement) 1e-4, relative
    gradient error 1e-4 for the traction field and the initial velocity."""
    sc, mesh, wc, _ = c5
    T50 = 50
    f, lw = _t(sc.f_ext), _t(sc.loss_w)

    def run(prec, tol, K):
        mesh.factorize(wc, None, None, None, h=sc.h, gravity=tuple(sc.gravity), precision=prec)
        o = api.solver_opts(tol_fwd=tol, tol_bwd=tol, max_iter_fwd=5000, max_iter_bwd=5000, checkpoint_every=K)
        r = mesh.forward(_t(sc.x0), _t(sc.v0), T50, f_ext=f, opts=o)
        g = mesh.backward(r, T50, lw, f_ext=f, opts=o, want=("fext", "v0"))
        return r.x[-1].cpu().numpy(), g["fext"].cpu().numpy(), g["v0"].cpu().numpy()
    x_ref, gf_ref, gv_ref = run(N.PD_PREC_FP64, 1e-10, 0)
    x, gf, gv = run(N.PD_PREC_MIXED, 1e-7, 25)
    d = x - x_ref
    u = x_ref - sc.x0
    pos = np.linalg.norm(d) / np.linalg.norm(x_ref)
    disp = np.linalg.norm(d) / np.linalg.norm(u)
    emax = np.abs(d).max() / np.abs(u).max()
    ef = np.linalg.norm(gf - gf_ref) / np.linalg.norm(gf_ref)
    ev = np.linalg.norm(gv - gv_ref) / np.linalg.norm(gv_ref)
    print(f"C5 50 steps, mixed tol 1e-7 vs FP64 tol 1e-10: position {pos:.2e}, displacement-relative {disp:.2e}, "
          f"max {emax:.2e}; grad f_ext {ef:.2e}, grad v0 {ev:.2e}")
    assert pos <= 1e-5 and disp <= 1e-4 and emax <= 1e-4
    assert ef <= 1e-4 and ev <= 1e-4
