"""Complementarity contact, global step with a fixed contact set (Sec. 5.2, Alg. 4):
the GPU low-rank update against the oracle's direct reduced solve, for empty,
single, ragged and full contact sets, in FP64 and mixed precision; argument checks."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import contact as oc
from oracle.model import Model
from oracle.pd_cpu import ScalarA
from paper_2101_05917_gb300 import _native as N
from paper_2101_05917_gb300 import api
from workloads import contact_cube_c3, napkin, quadruped, small_beam

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def _cases():
    beam = small_beam(5, 3, 4, T=1, traction=False)
    # beam candidates: bottom-face nodes (z = 0 plane of the grid), fixed ones excluded
    z = beam.x0[:, 2]
    beam_cand = (np.isclose(z, z.min()) & (beam.dirichlet == 0)).astype(np.uint8)
    cube = contact_cube_c3(N=6, T=1)
    quad = quadruped(8, T=1)
    # napkin: 169 bottom candidates; sets of 33, 97 and 169 nodes span several 32-column
    # blocks and 64-row tiles of the dense factorisation of S, with ragged tails
    nap = napkin(12, 0.5)
    return [("beam", beam, beam_cand), ("cube", cube, cube.contact.astype(np.uint8)),
            ("quadruped", quad, quad.contact.astype(np.uint8)), ("napkin", nap, nap.contact.astype(np.uint8))]


def _mesh(sc, precision):
    sc0 = dataclasses.replace(sc, k_contact=0.0)   # no penalty term in A
    mesh = api.PDMesh.from_scene(sc0)
    wc, wv, wm, fib = api.scene_weights(sc0, DEV)
    mesh.factorize(wc, wv, wm, fib, h=sc0.h, gravity=tuple(sc0.gravity), k_contact=0.0, precision=precision)
    L = ScalarA(Model(sc0)).LA
    return sc0, mesh, L


# mixed: the FP32 solve's ~1e-7 error is amplified by the correction when a large
# contact set cancels most of a1 (4e-5 with every surface node of the quadruped fixed)
@pytest.mark.parametrize("precision,tol", [(N.PD_PREC_FP64, 1e-10), (N.PD_PREC_MIXED, 1e-4)])
@pytest.mark.parametrize("case", range(4))
def test_constrained_solve_matches_oracle(precision, tol, case):
    name, sc, cand = _cases()[case]
    sc0, mesh, L = _mesh(sc, precision)
    mesh.contact_prepare(cand)
    free = np.flatnonzero(sc0.dirichlet == 0)
    pos_in_free = -np.ones(sc0.x0.shape[0], dtype=np.int64)
    pos_in_free[free] = np.arange(free.size)
    cands = np.flatnonzero(cand)
    rng = np.random.default_rng(100 + case)
    for c in sorted({0, 1, 7, 33, 97, cands.size} & set(range(cands.size + 1))):
        C = np.sort(rng.choice(cands, size=c, replace=False)) if c else np.zeros(0, dtype=np.int64)
        rng.shuffle(C)   # any order
        b = rng.standard_normal(sc0.x0.shape)
        xs = rng.standard_normal((c, 3))
        mesh.contact_set(C)
        x = mesh.solve_contact(_t(b), _t(xs) if c else None, precision=precision).cpu().numpy()
        ref = np.zeros_like(b)
        ref[free] = oc.constrained_solve(L, pos_in_free[C], xs, b[free])
        solved = np.setdiff1d(free, C)   # the rows the reduced system determines
        err = np.abs(x[solved] - ref[solved]).max() / np.abs(ref[solved]).max()
        assert not x[sc0.dirichlet != 0].any()
        print(f"{name} c={c} prec={precision}: max rel err {err:.2e}")
        assert err <= tol, (name, c, err)
        if c:
            assert np.array_equal(x[C], xs)
    mesh.close()


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def test_contact_argument_checks():
    name, sc, cand = _cases()[1]
    sc0, mesh, L = _mesh(sc, N.PD_PREC_FP64)
    with pytest.raises(N.PDError):
        mesh.contact_set([0])                    # before pd_contact_prepare
    mesh.contact_prepare(cand)
    non_cand = int(np.flatnonzero(cand == 0)[0])
    with pytest.raises(N.PDError):
        mesh.contact_set([non_cand])             # not a candidate
    c0 = int(np.flatnonzero(cand)[0])
    with pytest.raises(N.PDError):
        mesh.contact_set([c0, c0])               # repeated
    wc, wv, _, _ = api.scene_weights(sc0, DEV)
    mesh.factorize(wc * 2, wv, None, None, h=sc0.h, gravity=tuple(sc0.gravity))
    with pytest.raises(N.PDError):
        mesh.contact_set([c0])                   # candidate columns of the old factor
    mesh.close()
