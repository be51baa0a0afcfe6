"""The C ABI library loads, exports every symbol of include/diffpd.h, and its
host-side index construction reproduces the oracle's re-derivation bit for
bit (no GPU needed: meshes are created with device = -1)."""
import re

import numpy as np
import pytest

from oracle import structure
from workloads import cantilever_c1, quadruped, small_beam, contact_cube_c3, tet_ball


@pytest.fixture(scope="module")
def native():
    from paper_2101_05917_gb300 import build
    build.build()
    from paper_2101_05917_gb300 import _native
    return _native


def test_exports_every_declared_symbol(native):
    import os
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "diffpd.h")).read()
    declared = set(re.findall(r"\b(pd_[a-z_A]+)\s*\(", hdr))
    declared -= {"pd_status"}
    L = native.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(native.SYMBOLS)


CASES = [(cantilever_c1(), 64), (cantilever_c1(), 8), (quadruped(8, T=1), 16), (quadruped(9, T=1), 64),
         (small_beam(5, 3, 4, T=1), 5), (contact_cube_c3(N=6, T=1), 32), (tet_ball(T=1), 16)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_index_structures_bit_exact(native, case):
    from paper_2101_05917_gb300 import api
    sc, leaf = CASES[case]
    m = api.PDMesh.from_scene(sc, leaf_max=leaf, device=None)
    st = structure.analyse(sc.nx, sc.ny, sc.nz, sc.cell_mask, sc.dirichlet, leaf)
    for key in ("perm", "snode_first", "row_ptr", "rows", "parent", "level", "rel", "inc_ptr", "inc"):
        assert np.array_equal(m.export(key), st[key]), key
    assert np.array_equal(m.export("level_list"), np.concatenate(st["level_lists"]))
    lp = np.concatenate([[0], np.cumsum([len(l) for l in st["level_lists"]])])
    assert np.array_equal(m.export("level_ptr"), lp)
    m.close()


def test_invalid_arguments_are_rejected(native):
    from paper_2101_05917_gb300 import api, _native as N
    with pytest.raises(N.PDError):
        api.PDMesh(0, 1, 1, 0.01, 1e3, device=None)
    with pytest.raises(N.PDError):
        api.PDMesh(1, 1, 1, -0.01, 1e3, device=None)
    # every node fixed
    with pytest.raises(N.PDError):
        api.PDMesh(1, 1, 1, 0.01, 1e3, dirichlet=np.ones(8, np.uint8), device=None)
    # unknown element rule (binding and host analysis)
    with pytest.raises(ValueError):
        api.PDMesh(2, 1, 1, 0.01, 1e3, device=None, element_rule="hex27")
    import ctypes
    desc = N.MeshDesc()
    desc.nx, desc.ny, desc.nz, desc.dx, desc.density, desc.device, desc.element_rule = 2, 1, 1, 0.01, 1e3, -1, 7
    h = ctypes.c_void_p()
    assert N.lib().pd_create_mesh(ctypes.byref(desc), ctypes.byref(h)) == N.PD_ERR_INVALID_ARG
    m = api.PDMesh(2, 1, 1, 0.01, 1e3, device=None)
    import ctypes
    st = native.lib().pd_factorize(m.handle, None, None, None, None, None, None)
    assert st == N.PD_ERR_NO_DEVICE
    m.close()


def test_serve_create_rejects_bad_arguments(native):
    import ctypes
    import torch
    from paper_2101_05917_gb300 import _native as N
    L = native.lib()
    h = ctypes.c_void_p()
    assert L.pd_serve_create(0, 1 << 30, 0, ctypes.byref(h)) == N.PD_ERR_INVALID_ARG
    assert L.pd_serve_create(0, 1 << 30, 65, ctypes.byref(h)) == N.PD_ERR_INVALID_ARG
    assert not h.value
    if not torch.cuda.is_available():
        assert L.pd_serve_create(0, 1 << 30, 2, ctypes.byref(h)) == N.PD_ERR_NO_DEVICE
        assert not h.value
    assert L.pd_serve_submit(None, None, None) == N.PD_ERR_INVALID_ARG
    assert L.pd_serve_drain(None) == N.PD_ERR_INVALID_ARG


def test_serving_refuses_tetrahedral_scenes(native):
    from paper_2101_05917_gb300 import api
    from workloads import tet_beam
    srv = api.PDServer.__new__(api.PDServer)   # no device needed: the check comes first
    srv.handle = None
    with pytest.raises(ValueError):
        srv.submit_scene(tet_beam(2, 1, 1, T=1))


def test_backward_rejects_mismatched_loss_gradients(native):
    """pd_backward reads loss_states blocks of (n, 3): the Python front end checks
    the caller's shapes (states, loss gradients) and the C ABI refuses a
    loss_states that is neither 1 nor T+1 before it touches any array."""
    import ctypes
    import torch
    from paper_2101_05917_gb300 import api
    sc = small_beam(3, 2, 2, T=1)
    m = api.PDMesh.from_scene(sc, device=None)
    n, T, K = m.n, 4, 2
    opts = api.solver_opts(checkpoint_every=K)
    roll = api.Rollout(torch.zeros((T // K + 1, n, 3), dtype=torch.float64),
                       torch.zeros((T // K + 1, n, 3), dtype=torch.float64), {}, 0)
    # the checkpointed states' gradient where every state's is expected
    with pytest.raises(ValueError, match="dL_dx"):
        m.backward(roll, T, torch.zeros((T // K + 1, n, 3), dtype=torch.float64), loss_all_steps=True, opts=opts)
    with pytest.raises(ValueError, match="dL_dv"):
        m.backward(roll, T, torch.zeros((n, 3), dtype=torch.float64),
                   dL_dv=torch.zeros((T + 1, n, 3), dtype=torch.float64), opts=opts)
    # states stored for another checkpoint interval
    with pytest.raises(ValueError, match="rollout states"):
        m.backward(roll, T, torch.zeros((n, 3), dtype=torch.float64), opts=api.solver_opts())
    L = native.lib()
    for bad in (2, T, T + 2, -1):
        st = L.pd_backward(m.handle, None, None, None, None, 0.0, T, None, None, bad, None, None, None, None, None,
                           None, None, None, None, None, None)
        assert st == native.PD_ERR_INVALID_ARG
        assert b"loss_states" in L.pd_last_error()
    m.close()


def test_checkpoint_plan_follows_the_memory_cap(native):
    """pd_plan_checkpoints: every state stored when (T+1) states of x and v fit the
    cap; otherwise the smallest K dividing T whose checkpoints plus one recomputed
    segment fit; PD_ERR_OOM when none does (host arithmetic, no device)."""
    from paper_2101_05917_gb300 import api
    sc = small_beam(3, 2, 2, T=1)
    m = api.PDMesh.from_scene(sc, device=None)
    state = 48 * m.n                      # x and v of one state, bytes
    T = 12
    assert m.plan_checkpoints(T, (T + 1) * state) == 0
    # K fits when (T/K + 1) + (K + 1) states fit: 12 states -> K = 2 (6+1+2+1 = 10),
    # 9 states -> K = 3 (4+1+3+1 = 9), 8 states -> none (K = 3, 4, 6, 12 need 9, 9, 10, 15)
    assert m.plan_checkpoints(T, 9 * state) == 3
    assert m.plan_checkpoints(T, 12 * state) == 2
    with pytest.raises(native.PDError):
        m.plan_checkpoints(T, 8 * state)
    with pytest.raises(native.PDError):   # host-only mesh: the cap is required
        m.plan_checkpoints(T, 0)
    m.close()


def test_fext_layout_from_shape():
    """The Python front end sets fext_per_step from f_ext's shape ((n, 3) or
    (T, n, 3)) on a copy of the caller's options and rejects other shapes."""
    import torch
    from paper_2101_05917_gb300 import api
    o = api.solver_opts()
    n, T = 7, 4
    assert api._with_fext_layout(o, None, T, n).fext_per_step == 0
    assert api._with_fext_layout(o, torch.zeros((n, 3)), T, n).fext_per_step == 0
    p = api._with_fext_layout(o, torch.zeros((T, n, 3)), T, n)
    assert p.fext_per_step == 1 and o.fext_per_step == 0
    for bad in ((T + 1, n, 3), (n, 2), (T, n)):
        with pytest.raises(ValueError):
            api._with_fext_layout(o, torch.zeros(bad), T, n)
