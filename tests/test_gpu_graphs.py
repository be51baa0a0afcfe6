"""Iteration chunks replayed as CUDA graphs give bit-identical results to the
same kernels launched one by one (forward and adjoint, both precisions, with
actuation and contact)."""
import numpy as np
import pytest
import torch

from paper_2101_05917_gb300 import _native as N
from paper_2101_05917_gb300 import api
from workloads import quadruped, small_beam

pytestmark = pytest.mark.gpu


def _run(sc, T, precision, graphs, stream=None):
    dev = torch.device("cuda:0")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    mesh = api.PDMesh.from_scene(sc)
    wc, wv, wm, fib = api.scene_weights(sc, dev)
    mesh.factorize(wc, wv, wm, fib, h=sc.h, gravity=tuple(sc.gravity), k_contact=sc.k_contact,
                   precision=precision, stream=stream)
    opts = api.solver_opts(tol_fwd=1e-9, tol_bwd=1e-9, max_iter_fwd=3000, max_iter_bwd=3000, graphs=graphs)
    act = t(sc.act[:T]) if sc.act is not None else None
    roll = mesh.forward(t(sc.x0), t(sc.v0), T, f_ext=t(sc.f_ext), act=act, mu=sc.mu, opts=opts, stream=stream)
    g = mesh.backward(roll, T, t(sc.loss_w), f_ext=t(sc.f_ext), act=act, mu=sc.mu, opts=opts, stream=stream)
    torch.cuda.synchronize()
    mesh.close()
    return roll, g


@pytest.mark.parametrize("precision", [N.PD_PREC_MIXED, N.PD_PREC_FP64])
@pytest.mark.parametrize("which", ["beam", "quadruped"])
def test_graphs_bit_identical(precision, which):
    sc = small_beam(6, 3, 3, T=4) if which == "beam" else quadruped(5, T=3)
    T = sc.T
    a_roll, a_g = _run(sc, T, precision, graphs=True)
    b_roll, b_g = _run(sc, T, precision, graphs=False)
    assert torch.equal(a_roll.x, b_roll.x) and torch.equal(a_roll.v, b_roll.v)
    for k in b_g:
        if k != "stats":
            assert torch.equal(a_g[k], b_g[k]), k
    assert a_roll.stats["fwd_iters"] == b_roll.stats["fwd_iters"]
    assert a_roll.stats["kernel_launches"] == b_roll.stats["kernel_launches"]


def test_graphs_on_a_side_stream():
    sc = small_beam(5, 3, 3, T=3)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a_roll, a_g = _run(sc, sc.T, N.PD_PREC_MIXED, graphs=True, stream=s)
    b_roll, b_g = _run(sc, sc.T, N.PD_PREC_MIXED, graphs=False)
    assert torch.equal(a_roll.x, b_roll.x)
    assert torch.equal(a_g["v0"], b_g["v0"])
