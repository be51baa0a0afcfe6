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
