"""Complementarity contact through time (Sec. 5.2, Alg. 3 forward, Alg. 5
backward): a cube falling onto the ground, GPU against the oracle's active-set
Newton rollout and its adjoint (positions, contact sets, gradients)."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import contact as oc
from oracle.model import Model
from paper_2101_05917_gb300 import _native as N
from paper_2101_05917_gb300 import api
from workloads import contact_cube_c3

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def falling_cube(N=4, gap=0.002, vz=-0.6):
    sc = contact_cube_c3(N=N, T=4)
    x0 = sc.x0.copy()
    x0[:, 2] += gap - x0[:, 2].min()
    v0 = sc.v0 * 0.1
    v0[:, 2] += vz
    return dataclasses.replace(sc, x0=x0, v0=v0, k_contact=0.0, mu=0.0)


def _gpu(sc, T, precision, tol, want=None):
    mesh = api.PDMesh.from_scene(sc)
    wc, wv, _, _ = api.scene_weights(sc, DEV)
    mesh.factorize(wc, wv, None, None, h=sc.h, gravity=tuple(sc.gravity), k_contact=0.0, precision=precision)
    mesh.contact_prepare(sc.contact.astype(np.uint8))
    opts = api.solver_opts(tol_fwd=tol, tol_bwd=tol, max_iter_fwd=5000, max_iter_bwd=5000, complementarity=True)
    roll = mesh.forward(_t(sc.x0), _t(sc.v0), T, f_ext=_t(sc.f_ext), opts=opts)
    out = None
    if want:
        out = mesh.backward(roll, T, _t(sc.loss_w), f_ext=_t(sc.f_ext), opts=opts, want=want)
    return mesh, roll, out


@pytest.mark.parametrize("precision,tol,gate", [(N.PD_PREC_FP64, 1e-11, 1e-9), (N.PD_PREC_MIXED, 1e-9, 1e-6)])
def test_forward_matches_oracle(precision, tol, gate):
    sc = falling_cube()
    T = 4
    xs, vs, infos = oc.rollout_complementarity(Model(sc), sc.x0, sc.v0, sc.f_ext, sc.contact, T)
    mesh, roll, _ = _gpu(sc, T, precision, tol)
    xg = roll.x.cpu().numpy()
    for t in range(1, T + 1):
        err = np.linalg.norm(xg[t] - xs[t]) / np.linalg.norm(xs[t] - sc.x0)
        contact_gpu = int(np.sum(np.isclose(xg[t][:, 2], 0.0, atol=1e-12) & (sc.contact > 0)))
        print(f"step {t}: displacement-relative position error {err:.2e}, contact set {infos[t - 1]['C'].size} "
              f"(ground nodes gpu {contact_gpu})")
        assert err <= gate
    mesh.close()
