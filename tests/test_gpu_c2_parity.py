"""Full-size parity on the 32x32x64 beam (212,355 DoFs) in the configuration the
benchmark times (mixed precision, tol 1e-7, L-BFGS m = 5): the first two steps
and their adjoint against the FP64 oracle stored by tests/golden/make_golden.py
(PD + L-BFGS polished to 1e-12 and an A^-1-preconditioned MINRES adjoint, on
2000 sampled nodes and cells).  Gates: 1e-5 relative position error and 1e-4
relative gradient error."""
import os

import numpy as np
import pytest
import torch

from paper_2101_05917_gb300 import _native as N
from paper_2101_05917_gb300 import api
from workloads import beam_c2

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "c2_beam_T2_oracle_sampled.npz")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("lbfgs_m", [5, 10])
def test_c2_first_steps_match_oracle(lbfgs_m):
    g = np.load(GOLD)
    T = int(g["T"])
    sc = beam_c2(T=T)
    dev = torch.device("cuda:0")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    mesh = api.PDMesh.from_scene(sc)
    wc, wv, wm, fib = api.scene_weights(sc, dev)
    mesh.factorize(wc, wv, wm, fib, h=sc.h, gravity=tuple(sc.gravity), precision=N.PD_PREC_MIXED)
    opts = api.solver_opts(tol_fwd=1e-7, tol_bwd=1e-7, lbfgs_m=lbfgs_m, max_iter_fwd=3000, max_iter_bwd=3000)
    roll = mesh.forward(t(sc.x0), t(sc.v0), T, f_ext=t(sc.f_ext), opts=opts)
    out = mesh.backward(roll, T, t(sc.loss_w), f_ext=t(sc.f_ext), opts=opts, want=("v0", "w_corot", "w_vol"))
    nodes, cells = g["nodes"], g["cells"]
    xs = roll.x.cpu().numpy()[:, nodes]
    X = sc.x0[nodes]
    pos = max(_rel(xs[k], g["xs"][k]) for k in range(1, T + 1))
    disp = max(np.linalg.norm(xs[k] - g["xs"][k]) / np.linalg.norm(g["xs"][k] - X) for k in range(1, T + 1))
    gv0 = _rel(out["v0"].cpu().numpy()[nodes], g["g_v0"])
    gwc = _rel(out["w_corot"].cpu().numpy()[cells], g["g_wc"])
    gwv = _rel(out["w_vol"].cpu().numpy()[cells], g["g_wv"])
    print(f"m={lbfgs_m} position {pos:.2e} (displacement-relative {disp:.2e}) grad v0 {gv0:.2e} "
          f"w_corot {gwc:.2e} w_vol {gwv:.2e}")
    assert pos <= 1e-5
    assert max(gv0, gwc, gwv) <= 1e-4
    mesh.close()
