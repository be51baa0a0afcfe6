"""Failure detection without a GPU fault: inputs the library must reject or flag,
each ending in a status the host reads (never a trap, a fault or a hang), after
which the same mesh still works.  Non-finite state (PD_ERR_NAN), a matrix A that
is not SPD (PD_ERR_NOT_SPD from the factorisation's pivots), an inverted element
(det F <= 0, flagged in the statistics; Sec. 3's signed polar projection keeps the
step finite) and the iteration cap (PD_ERR_NOT_CONVERGED with valid outputs)."""
import numpy as np
import pytest
import torch

from _gpu_helpers import DEV, T, make_mesh
from paper_2101_05917_gb300 import api
from paper_2101_05917_gb300 import _native as N
from workloads import small_beam

pytestmark = pytest.mark.gpu

OPTS = dict(tol_fwd=1e-10, tol_bwd=1e-10)


def _forward(mesh, sc, x0, **kw):
    return mesh.forward(T(x0), T(sc.v0), sc.T, f_ext=T(sc.f_ext), **kw)


def test_non_finite_state_returns_nan_status():
    sc = small_beam(3, 2, 2, T=3)
    mesh = make_mesh(sc)
    x0 = sc.x0.copy()
    x0[-1, 1] = np.nan                      # a free node (the x = 0 face is fixed)
    with pytest.raises(N.PDError) as err:
        _forward(mesh, sc, x0, opts=api.solver_opts(**OPTS))
    assert err.value.status == N.PD_ERR_NAN
    roll = _forward(mesh, sc, sc.x0, opts=api.solver_opts(**OPTS))
    torch.cuda.synchronize()
    assert roll.status == N.PD_OK and np.all(np.isfinite(roll.x.cpu().numpy()))
    mesh.close()


def test_matrix_that_is_not_spd_is_reported():
    sc = small_beam(3, 2, 2, T=2)
    mesh = api.PDMesh.from_scene(sc)
    wc, wv, wm, fib = api.scene_weights(sc, DEV)
    # a negative stiffness far above the mass term makes A indefinite
    with pytest.raises(N.PDError) as err:
        mesh.factorize(-10.0 * wc, None, None, None, h=sc.h, gravity=tuple(sc.gravity))
    assert err.value.status == N.PD_ERR_NOT_SPD
    # no rollout on the failed factor; a valid factorisation afterwards works
    with pytest.raises(N.PDError):
        _forward(mesh, sc, sc.x0, opts=api.solver_opts(**OPTS))
    mesh.factorize(wc, wv, wm, fib, h=sc.h, gravity=tuple(sc.gravity))
    roll = _forward(mesh, sc, sc.x0, opts=api.solver_opts(**OPTS))
    torch.cuda.synchronize()
    assert roll.status == N.PD_OK and np.all(np.isfinite(roll.x.cpu().numpy()))
    mesh.close()


def test_inverted_element_is_flagged():
    sc = small_beam(3, 2, 2, T=1, volume=False)
    mesh = make_mesh(sc)
    ok = _forward(mesh, sc, sc.x0, opts=api.solver_opts(**OPTS))
    assert ok.stats["inverted"] == 0
    # push the far corner node through the opposite face of its cell
    x0 = sc.x0.copy()
    x0[-1, 0] -= 3.0 * sc.dx   # F_xx at the nearest Gauss point: 1 - 3 (0.789)^2 < 0
    roll = _forward(mesh, sc, x0, opts=api.solver_opts(max_iter_fwd=20, max_iter_bwd=20, **OPTS),
                    allow_not_converged=True)
    torch.cuda.synchronize()
    assert roll.stats["inverted"] == 1
    assert roll.status in (N.PD_OK, N.PD_ERR_NOT_CONVERGED)
    assert np.all(np.isfinite(roll.x.cpu().numpy()))
    mesh.close()


def test_iteration_cap_reports_not_converged():
    sc = small_beam(3, 2, 2, T=2)
    mesh = make_mesh(sc)
    capped = api.solver_opts(tol_fwd=1e-14, tol_bwd=1e-14, max_iter_fwd=2, max_iter_bwd=2)
    with pytest.raises(N.PDError) as err:
        _forward(mesh, sc, sc.x0, opts=capped)
    assert err.value.status == N.PD_ERR_NOT_CONVERGED
    roll = _forward(mesh, sc, sc.x0, opts=capped, allow_not_converged=True)
    torch.cuda.synchronize()
    assert roll.status == N.PD_ERR_NOT_CONVERGED
    assert roll.stats["not_converged_steps"] == sc.T
    assert np.all(np.isfinite(roll.x.cpu().numpy()))
    mesh.close()


@pytest.mark.parametrize("prec", [N.PD_PREC_FP64, N.PD_PREC_MIXED])
def test_solve_dependency_wait_runs_out(monkeypatch, prec):
    """A bounded device wait that gives up reports PD_ERR_TIMEOUT instead of
    hanging.  The test hook PD_TEST_SOLVE_STALLS=1 makes the first solve of the
    mesh wait for one forward block more than its children deliver (nothing
    else is changed), with the wait bound lowered to 20,000 polls by
    PD_SOLVE_SPIN_LIMIT; the wait runs out, the call returns the status, and
    the next solve on the same mesh is correct."""
    from oracle.model import Model
    sc = small_beam(6, 3, 3, T=1)
    monkeypatch.setenv("PD_SOLVE_SPIN_LIMIT", "20000")
    monkeypatch.setenv("PD_TEST_SOLVE_STALLS", "1")
    mesh = make_mesh(sc, precision=prec, leaf_max=8)   # several levels: the root waits for children
    monkeypatch.delenv("PD_TEST_SOLVE_STALLS")
    model = Model(sc)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(sc.x0.shape)
    b[model.dirichlet] = 0
    with pytest.raises(N.PDError) as err:
        mesh.solve(T(b), precision=prec)
    assert err.value.status == N.PD_ERR_TIMEOUT
    x = mesh.solve(T(b), precision=prec).cpu().numpy()
    A = model.A_matrix().toarray() if hasattr(model.A_matrix(), "toarray") else model.A_matrix()
    fd = model.free_dofs
    ref = np.zeros(b.size)
    ref[fd] = np.linalg.solve(A[np.ix_(fd, fd)], b.ravel()[fd])
    tol = 1e-10 if prec == N.PD_PREC_FP64 else 2e-5
    assert np.linalg.norm(x.ravel() - ref) <= tol * np.linalg.norm(ref)
    # the rollout path on the same mesh works too
    roll = _forward(mesh, sc, sc.x0, opts=api.solver_opts(**OPTS))
    assert roll.status == N.PD_OK
    mesh.close()
