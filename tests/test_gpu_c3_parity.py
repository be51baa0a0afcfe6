"""Full-size contact cube (24^3 cells, 46,875 DoFs, penalty ground contact on 3,458
surface nodes, friction; Sec. 5.1) against the stored Newton oracle with the
full-linearisation adjoint (tests/golden/make_golden.py): positions and gradients
w.r.t. v0 and x0 on 2000 sampled nodes, the loss, and the friction-coefficient
gradient, in FP64 and mixed precision."""
import os

import numpy as np
import pytest
import torch

from paper_2101_05917_gb300 import _native as N
from paper_2101_05917_gb300 import api
from workloads import contact_cube_c3

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def _run(fname, precision, tol):
    path = os.path.join(HERE, fname)
    if not os.path.exists(path):
        pytest.skip(f"{fname} not generated")
    g = np.load(path)
    T = int(g["T"])
    sc = contact_cube_c3(T=T)
    dev = torch.device("cuda:0")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    mesh = api.PDMesh.from_scene(sc)
    wc, wv, _, _ = api.scene_weights(sc, dev)
    mesh.factorize(wc, wv, None, None, h=sc.h, gravity=tuple(sc.gravity), k_contact=sc.k_contact,
                   precision=precision)
    opts = api.solver_opts(tol_fwd=tol, tol_bwd=tol, max_iter_fwd=5000, max_iter_bwd=5000)
    roll = mesh.forward(t(sc.x0), t(sc.v0), T, f_ext=t(sc.f_ext), mu=sc.mu, opts=opts)
    out = mesh.backward(roll, T, t(sc.loss_w), f_ext=t(sc.f_ext), mu=sc.mu, opts=opts, want=("x0", "v0", "mu"))
    nodes = g["nodes"]
    xs = roll.x.cpu().numpy()
    pos = max(_rel(xs[k][nodes], g["xs"][k]) for k in range(1, T + 1))
    gv0 = _rel(out["v0"].cpu().numpy()[nodes], g["g_v0"])
    gx0 = _rel(out["x0"].cpu().numpy()[nodes], g["g_x0"])
    loss = float(np.sum(sc.loss_w * xs[-1]))
    gmu = float(out["mu"].cpu().numpy()[0])
    contact = int(np.sum((xs[-1][:, 2] < 0) & (sc.contact > 0)))
    print(f"{fname} prec={precision} position {pos:.2e} grad v0 {gv0:.2e} x0 {gx0:.2e} loss {loss:.12e} "
          f"(oracle {float(g['loss']):.12e}) g_mu {gmu:.6e} (oracle {float(g['g_mu']):.6e}) contact nodes {contact}")
    mesh.close()
    return g, pos, gv0, gx0, loss, gmu, contact


@pytest.mark.parametrize("precision,tol", [(N.PD_PREC_FP64, 1e-10), (N.PD_PREC_MIXED, 1e-7)])
def test_c3_first_steps(precision, tol):
    g, pos, gv0, gx0, loss, gmu, contact = _run("c3_cube_T2_oracle_sampled.npz", precision, tol)
    assert pos <= 1e-5
    assert max(gv0, gx0) <= 1e-4
    assert abs(loss - float(g["loss"])) <= 1e-5 * abs(float(g["loss"]))
    assert contact == int(g["contact_nodes"][-1])


@pytest.mark.parametrize("precision,tol", [(N.PD_PREC_FP64, 1e-10), (N.PD_PREC_MIXED, 1e-7)])
def test_c3_through_first_contact(precision, tol):
    g, pos, gv0, gx0, loss, gmu, contact = _run("c3_cube_T24_oracle_sampled.npz", precision, tol)
    assert int(g["contact_nodes"][-1]) > 0          # the horizon reaches the ground
    assert contact == int(g["contact_nodes"][-1])
    assert pos <= 1e-5
    assert max(gv0, gx0) <= 1e-4
    # every contact node is in the static friction regime here (m |v_t| / h < mu f_n),
    # where the friction force does not depend on mu: both sides give 0
    assert abs(gmu - float(g["g_mu"])) <= 1e-4 * abs(float(g["g_mu"])) + 1e-12
