"""The allocation-free local step (pd_local_step_noalloc) against pd_local_step
and the FP64 oracle.

pd_local_step_noalloc exists for callers that cannot allocate device memory
(under a device-memory budget fixed in advance, or behind an allocator the
library cannot reach): it takes every array from the caller and keeps its
scratch in one fixed device array inside the library.  This test calls it
through the C ABI twice in a row on the same inputs and compares both results
with the regular entry point, which owns its workspace, and with the oracle's
grad E and energy, within the tolerances of the other kernel parity tests; it
reads the status word back (clear on a regular state, the det F <= 0 bit on an
inverted cell) and checks that oversized meshes are refused.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle.model import Model
from paper_2101_05917_gb300 import api
from paper_2101_05917_gb300 import _native as N
from workloads import grid_node_ids, kept_nodes, small_beam

pytestmark = pytest.mark.gpu

TOL = {N.PD_PREC_FP64: 1e-10, N.PD_PREC_MIXED: 2e-5}


def _contact_scene():
    from test_oracle_dynamics import tiny_everything_scene
    return tiny_everything_scene()


def _kept_elems(sc):
    corners = grid_node_ids(sc.nx, sc.ny, sc.nz)
    if sc.cell_mask is not None:
        corners = corners[np.asarray(sc.cell_mask, dtype=bool)]
    nodes = kept_nodes(sc.nx, sc.ny, sc.nz, sc.cell_mask)
    return np.searchsorted(nodes, corners).astype(np.int32)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("name", ["beam_vol", "contact_muscle"])
@pytest.mark.parametrize("prec", [N.PD_PREC_FP64, N.PD_PREC_MIXED])
def test_noalloc_local_step_matches_regular_entry_point(name, prec):
    sc = small_beam(5, 3, 4, T=1) if name == "beam_vol" else _contact_scene()
    dev = torch.device("cuda:0")
    mesh = api.PDMesh.from_scene(sc, device=0)
    wc, wv, wm, fib = api.scene_weights(sc, dev)
    mesh.factorize(wc, wv, wm, fib, h=sc.h, gravity=tuple(sc.gravity), k_contact=sc.k_contact, precision=prec)
    rng = np.random.default_rng(5)
    x = sc.x0 + 0.05 * sc.dx * rng.standard_normal(sc.x0.shape)
    if sc.k_contact > 0:
        x[:, 2] -= 0.3 * sc.dx
    xt = torch.as_tensor(x, dtype=torch.float64, device=dev)
    act = None if sc.act is None else torch.as_tensor(sc.act[0], dtype=torch.float64, device=dev)
    g_ref, e_ref = mesh.local_step(xt, act, precision=prec)

    elems = torch.as_tensor(_kept_elems(sc), device=dev)
    inc_ptr = torch.as_tensor(mesh.export("inc_ptr").astype(np.int32), device=dev)
    inc = torch.as_tensor(mesh.export("inc").astype(np.int32), device=dev)
    contact = (torch.as_tensor(np.asarray(sc.contact, dtype=np.uint8), device=dev)
               if sc.k_contact > 0 else None)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    model = Model(sc)
    g_or = model.grad_E(x, None if sc.act is None else sc.act[0])
    e_or = model.energy(x, None if sc.act is None else sc.act[0])
    for _ in range(2):
        g = torch.full((mesh.n, 3), np.nan, dtype=torch.float64, device=dev)
        e = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        flags = torch.full((1,), -1, dtype=torch.int32, device=dev)
        st = N.lib().pd_local_step_noalloc(mesh.n, mesh.e, _ptr(elems), _ptr(inc_ptr), _ptr(inc), sc.dx, _ptr(xt),
                                           _ptr(act), _ptr(wc), _ptr(wv), _ptr(wm), _ptr(fib), _ptr(contact),
                                           sc.k_contact, prec, _ptr(g), _ptr(e), _ptr(flags), stream)
        N.check(st, "pd_local_step_noalloc")
        torch.cuda.synchronize()
        gr = g_ref.cpu().numpy()
        gn = g.cpu().numpy()
        assert np.linalg.norm(gn - gr) <= TOL[prec] * np.linalg.norm(gr)
        assert abs(e.item() - e_ref.item()) <= TOL[prec] * abs(e_ref.item())
        assert np.linalg.norm(gn - g_or) <= TOL[prec] * np.linalg.norm(g_or)
        assert abs(e.item() - e_or) <= TOL[prec] * abs(e_or)
        assert int(flags.item()) == 0
    mesh.close()


def test_noalloc_reports_inverted_cells():
    """A cell turned inside out (det F < 0) is a valid input: the gradient stays
    finite and the status word carries PD_LOCAL_FLAG_INVERTED, on two calls in a
    row (the word is cleared at the start of each call)."""
    sc = small_beam(3, 2, 2, T=1, volume=False)
    dev = torch.device("cuda:0")
    mesh = api.PDMesh.from_scene(sc, device=0)
    wc, _, _, _ = api.scene_weights(sc, dev)
    elems = torch.as_tensor(_kept_elems(sc), device=dev)
    inc_ptr = torch.as_tensor(mesh.export("inc_ptr").astype(np.int32), device=dev)
    inc = torch.as_tensor(mesh.export("inc").astype(np.int32), device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    x_rest = sc.x0.copy()
    x_inv = sc.x0.copy()
    x_inv[:, 2] = -x_inv[:, 2]          # mirror every cell: det F = -1
    for x, want in ((x_inv, 2), (x_rest, 0), (x_inv, 2)):
        xt = torch.as_tensor(x, dtype=torch.float64, device=dev)
        g = torch.full((mesh.n, 3), np.nan, dtype=torch.float64, device=dev)
        flags = torch.full((1,), -1, dtype=torch.int32, device=dev)
        st = N.lib().pd_local_step_noalloc(mesh.n, mesh.e, _ptr(elems), _ptr(inc_ptr), _ptr(inc), sc.dx, _ptr(xt),
                                           None, _ptr(wc), None, None, None, None, 0.0, N.PD_PREC_FP64,
                                           _ptr(g), None, _ptr(flags), stream)
        N.check(st, "pd_local_step_noalloc")
        torch.cuda.synchronize()
        assert int(flags.item()) == want
        assert np.isfinite(g.cpu().numpy()).all()
    mesh.close()


def test_noalloc_rejects_oversized_meshes():
    dev = torch.device("cuda:0")
    dummy = torch.zeros(8, dtype=torch.float64, device=dev)
    too_many = 32768 + 1
    st = N.lib().pd_local_step_noalloc(8, too_many, _ptr(dummy), _ptr(dummy), _ptr(dummy), 0.01, _ptr(dummy),
                                       None, _ptr(dummy), None, None, None, None, 0.0, N.PD_PREC_FP64,
                                       _ptr(dummy), None, None, None)
    assert st == N.PD_ERR_INVALID_ARG
    assert b"scratch" in N.lib().pd_last_error()
