"""Serving (pd_serve_*): results of a request do not depend on the other
requests running beside it, equal those of the direct entry points, and the
slot caches reuse meshes and factors without changing results."""
import numpy as np
import pytest
import torch

from paper_2101_05917_gb300 import _native as N
from paper_2101_05917_gb300 import api
from workloads import quadruped

pytestmark = pytest.mark.gpu

OPTS = dict(tol_fwd=1e-9, tol_bwd=1e-9, max_iter_fwd=3000, max_iter_bwd=3000)


def _scenes():
    return [quadruped(N, T=4, request=i) for i, N in enumerate([4, 5, 6, 4, 5, 6])]


def _same(a, b):
    assert a["status"] == b["status"] == N.PD_OK
    np.testing.assert_array_equal(a["x_final"], b["x_final"])
    np.testing.assert_array_equal(a["g_v0"], b["g_v0"])
    np.testing.assert_array_equal(a["g_act"], b["g_act"])
    assert a["loss"] == b["loss"]


@pytest.mark.parametrize("precision", [N.PD_PREC_MIXED, N.PD_PREC_FP64])
def test_alone_equals_mixed(precision):
    scenes = _scenes()
    opts = api.solver_opts(**OPTS)
    alone = []
    srv = api.PDServer(max_slots=1)
    for sc in scenes:
        alone.append(srv.result(srv.submit_scene(sc, precision=precision, opts=opts)))
    srv.close()
    srv = api.PDServer(max_slots=3)
    tickets = [srv.submit_scene(sc, precision=precision, opts=opts) for sc in scenes]
    mixed = [srv.result(t) for t in tickets]
    srv.close()
    assert len({r["slot"] for r in mixed}) > 1
    for a, b in zip(alone, mixed):
        _same(a, b)


def test_matches_direct_entry_points():
    sc = quadruped(5, T=4, request=3)
    opts = api.solver_opts(**OPTS)
    srv = api.PDServer(max_slots=2)
    r = srv.result(srv.submit_scene(sc, precision=N.PD_PREC_MIXED, opts=opts))
    srv.close()
    dev = torch.device("cuda:0")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    mesh = api.PDMesh.from_scene(sc)
    wc, wv, wm, fib = api.scene_weights(sc, dev)
    mesh.factorize(wc, wv, wm, fib, h=sc.h, gravity=tuple(sc.gravity), k_contact=sc.k_contact,
                   precision=N.PD_PREC_MIXED)
    act = t(sc.act[:4])
    roll = mesh.forward(t(sc.x0), t(sc.v0), 4, f_ext=t(sc.f_ext), act=act, mu=sc.mu, opts=opts)
    g = mesh.backward(roll, 4, t(sc.loss_w), f_ext=t(sc.f_ext), act=act, mu=sc.mu, opts=opts, want=("v0", "act"))
    np.testing.assert_array_equal(r["x_final"], roll.x[-1].cpu().numpy())
    np.testing.assert_array_equal(r["g_v0"], g["v0"].cpu().numpy())
    np.testing.assert_array_equal(r["g_act"], g["act"].cpu().numpy())
    assert abs(r["loss"] - float(np.sum(sc.loss_w * r["x_final"]))) <= 1e-12 * abs(r["loss"])


def test_cache_reuse_and_release():
    sc = quadruped(4, T=3, request=1)
    opts = api.solver_opts(**OPTS)
    srv = api.PDServer(max_slots=1)
    t1 = srv.submit_scene(sc, opts=opts)
    t2 = srv.submit_scene(sc, opts=opts)
    a, b = srv.result(t1), srv.result(t2)
    assert (a["mesh_cached"], a["factor_cached"]) == (0, 0)
    assert (b["mesh_cached"], b["factor_cached"]) == (1, 1)
    _same(a, b)
    # other materials on the cached mesh: refactorised, results change
    sc2 = quadruped(4, T=3, request=1)
    sc2.youngs = sc2.youngs * 1.5
    c = srv.result(srv.submit_scene(sc2, opts=opts))
    assert (c["mesh_cached"], c["factor_cached"]) == (1, 0)
    assert not np.array_equal(a["x_final"], c["x_final"])
    # another geometry key (fixed nodes) with the same box: a new mesh, compared in full
    sc3 = quadruped(4, T=3, request=1)
    sc3.dirichlet = sc3.dirichlet.copy()
    sc3.dirichlet[0] = 1
    d = srv.result(srv.submit_scene(sc3, opts=opts))
    assert d["mesh_cached"] == 0
    with pytest.raises(N.PDError):
        srv.poll(t1)            # released by result()
    with pytest.raises(N.PDError):
        srv.poll(10 ** 9)       # never issued
    srv.drain()
    srv.close()


def test_request_errors():
    srv = api.PDServer(max_slots=1)
    sc = quadruped(4, T=3)
    with pytest.raises(N.PDError):
        srv.submit_scene(sc, T=0)
    # iteration cap reached: the request's status says so, outputs are present
    r = srv.result(srv.submit_scene(sc, opts=api.solver_opts(tol_fwd=1e-14, max_iter_fwd=2, max_iter_bwd=2)))
    assert r["status"] == N.PD_ERR_NOT_CONVERGED
    assert r["x_final"] is not None and np.all(np.isfinite(r["x_final"]))
    srv.close()


def test_request_matches_newton_oracle():
    """One served request (quadruped with muscles, ground contact and friction, 3
    steps, mixed precision) against the FP64 oracle: Newton forward and the
    full-linearisation adjoint of L = sum(loss_w x_T) (Sec. 3, Sec. 4)."""
    from oracle import adjoint, newton
    from oracle.model import Model
    T = 3
    sc = quadruped(5, T=T, request=2)
    srv = api.PDServer(max_slots=2)
    r = srv.result(srv.submit_scene(sc, precision=N.PD_PREC_MIXED, opts=api.solver_opts(**OPTS)))
    srv.close()
    assert r["status"] == N.PD_OK
    model = Model(sc)
    act = sc.act[:T]
    xs, vs, _ = newton.rollout(model, sc.x0, sc.v0, sc.f_ext, act=act, mu=sc.mu, T=T)
    loss, gx = adjoint.final_position_loss(model, xs, sc.loss_w)
    g = adjoint.backward(model, xs, vs, gx, act=act, mu=sc.mu)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    disp = np.linalg.norm(r["x_final"] - xs[-1]) / np.linalg.norm(xs[-1] - sc.x0)
    print(f"served vs oracle: position {rel(r['x_final'], xs[-1]):.2e} (displacement-relative {disp:.2e}), "
          f"g_v0 {rel(r['g_v0'], g['g_v0']):.2e}, g_act {rel(r['g_act'], g['g_act']):.2e}")
    assert rel(r["x_final"], xs[-1]) <= 1e-5 and disp <= 1e-4
    assert rel(r["g_v0"], g["g_v0"]) <= 1e-4 and rel(r["g_act"], g["g_act"]) <= 1e-4
    assert abs(r["loss"] - loss) <= 1e-5 * abs(loss)


@pytest.mark.parametrize("budget", ["tiny", "large"])
def test_memory_budget_admission(budget):
    """Admission by device memory: with a budget below any request's estimate every
    request runs alone (a request that fits nowhere runs only when nothing else
    does), so their run intervals do not overlap; with a large budget three slots
    run them side by side.  Results are the same either way."""
    import time
    scenes = [quadruped(8, T=6, request=i) for i in range(3)]
    opts = api.solver_opts(**OPTS)
    srv = api.PDServer(max_slots=3, mem_budget=1 if budget == "tiny" else 16 << 30)
    subs, tickets = [], []
    for sc in scenes:
        subs.append(time.perf_counter())
        tickets.append(srv.submit_scene(sc, precision=N.PD_PREC_MIXED, opts=opts))
    res = [srv.result(t) for t in tickets]
    srv.close()
    spans = sorted((s + 1e-3 * r["queue_ms"], s + 1e-3 * r["latency_ms"]) for s, r in zip(subs, res))
    overlaps = sum(1 for a, b in zip(spans, spans[1:]) if b[0] < a[1] - 2e-3)
    if budget == "tiny":
        assert overlaps == 0, spans
    else:
        assert overlaps > 0, spans
    ref = api.PDServer(max_slots=1)
    for sc, r in zip(scenes, res):
        _same(r, ref.result(ref.submit_scene(sc, precision=N.PD_PREC_MIXED, opts=opts)))
    ref.close()
