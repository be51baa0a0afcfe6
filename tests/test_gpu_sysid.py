"""Optimisation through the simulator (Sec. 7 parameter estimation): L-BFGS on
log E and log nu recovers the parameters that generated an observed trajectory
of a cantilever (refactorising A at every evaluation)."""
import numpy as np
import pytest
import torch

from paper_2101_05917_gb300 import _native as N
from paper_2101_05917_gb300 import sysid
from paper_2101_05917_gb300.autograd import Simulator
from workloads import small_beam

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [N.PD_PREC_FP64, N.PD_PREC_MIXED])
def test_recovers_material_parameters(precision):
    sc = small_beam(8, 3, 3, T=12, e_sigma=0.0, v0_sigma=0.05, E=2e5)
    dev = torch.device("cuda:0")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    opts = dict(tol_fwd=1e-11, tol_bwd=1e-11, max_iter_fwd=5000, max_iter_bwd=5000)
    # the observation: the simulator's own trajectory at the true parameters
    true_logE, true_lognu = np.log(2e5), np.log(0.45)
    sim = Simulator.from_scene(sc, precision=N.PD_PREC_FP64, opts=opts)
    wc, wv = sysid._weights(t(np.full(sc.n_elems, true_logE)), torch.tensor(true_lognu, dtype=torch.float64,
                                                                             device=dev))
    with torch.no_grad():
        x_obs, _ = sim.rollout(t(sc.x0), t(sc.v0), sc.T, f_ext=t(sc.f_ext), w_corot=wc, w_vol=wv)
    sim.mesh.close()
    # start: E 49 % too stiff, nu 0.38 instead of 0.45
    res = sysid.identify(sc, x_obs, true_logE + 0.4, np.log(0.38), iters=40, precision=precision, opts=opts)
    print(f"prec {precision}: evaluations {res.evaluations}, loss {res.loss_history[0]:.3e} -> "
          f"{min(res.loss_history):.3e}, E {np.exp(res.log_E[0]):.6e}, nu {np.exp(res.log_nu):.6f}")
    assert min(res.loss_history) < 1e-10 * res.loss_history[0]
    assert abs(res.log_E[0] - true_logE) < 1e-5
    assert abs(res.log_nu - true_lognu) < 1e-5
