"""Python front end of the C ABI: device memory and streams come from PyTorch,
every step of the computation runs in libdiffpd.so."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import _native as N


def material_weights(E, nu):
    """Stiffness per unit volume of the corotated (2 mu) and volume-preserving
    (lambda) energies from Young's modulus and Poisson's ratio."""
    w_corot = E / (1.0 + nu)
    w_vol = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return w_corot, w_vol


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), "expected contiguous CUDA float64"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _u8(a, n, name):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.uint8).reshape(-1))
    if arr.size != n:
        raise ValueError(f"{name}: expected {n} entries, got {arr.size}")
    return arr, arr.ctypes.data_as(N.c_u8_p)


def solver_opts(tol_fwd=1e-9, tol_bwd=1e-9, max_iter_fwd=500, max_iter_bwd=500, lbfgs_m=5, ls_max=10,
                checkpoint_every=0, check_every=4, profile=False, warm_start=False, graphs=True,
                complementarity=False, step_ms: Optional[np.ndarray] = None,
                step_iters: Optional[np.ndarray] = None) -> N.SolverOpts:
    """checkpoint_every: 0 = every state stored, K > 0 = states 0, K, 2K, ..., -1 =
    planned by PDMesh.forward from its mem_cap (pd_plan_checkpoints).
    step_ms: optional float64 host array of T entries receiving the per-step
    wall time (forward, then the backward adds its own); step_iters: optional
    int32 host array of T entries receiving the per-step iterations (forward, then
    the backward's adjoint iterations); the caller keeps both alive."""
    p = None
    if step_ms is not None:
        assert step_ms.dtype == np.float64 and step_ms.flags.c_contiguous
        p = step_ms.ctypes.data_as(N.c_double_p)
    q = None
    if step_iters is not None:
        assert step_iters.dtype == np.int32 and step_iters.flags.c_contiguous
        q = step_iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    return N.SolverOpts(tol_fwd, tol_bwd, max_iter_fwd, max_iter_bwd, lbfgs_m, ls_max, checkpoint_every,
                        check_every, 1 if profile else 0, 1 if warm_start else 0, 0 if graphs else 1,
                        1 if complementarity else 0, p, q)


@dataclass
class Rollout:
    x: torch.Tensor      # (S, n, 3)
    v: torch.Tensor
    stats: dict
    status: int
    checkpoint_every: int = 0   # 0: every state stored; K: states 0, K, 2K, ...


def _with_fext_layout(opts, f_ext, T, n):
    """opts with fext_per_step set from the shape of f_ext ((n, 3) or (T, n, 3));
    the caller's opts are not modified."""
    per_step = f_ext is not None and f_ext.dim() == 3
    if f_ext is not None:
        want = (T, n, 3) if per_step else (n, 3)
        if tuple(f_ext.shape) != want:
            raise ValueError(f"f_ext: expected shape (n, 3) or (T, n, 3) = {(T, n, 3)}, got {tuple(f_ext.shape)}")
    if bool(opts.fext_per_step) == per_step:
        return opts
    o = N.SolverOpts.from_buffer_copy(opts)
    o.fext_per_step = 1 if per_step else 0
    return o


class PDMesh:
    """A voxel mesh (hexahedra, or six tetrahedra per cell with element_rule
    "tet6") or an unstructured tetrahedral mesh (from_tet_mesh) resident on one GPU
    (pd_create_mesh / pd_create_tet_mesh ... pd_mesh_destroy)."""

    def __init__(self, nx, ny, nz, dx, density, origin=(0.0, 0.0, 0.0), cell_mask=None, dirichlet=None,
                 contact=None, leaf_max=64, device: Optional[int] = 0, element_rule: str = "hex8"):
        L = N.lib()
        self._keep = []
        mask_arr, mask_p = _u8(cell_mask, nx * ny * nz, "cell_mask")
        desc = N.MeshDesc()
        desc.nx, desc.ny, desc.nz = nx, ny, nz
        desc.dx = dx
        desc.origin = (ctypes.c_double * 3)(*origin)
        desc.density = density
        desc.cell_mask = mask_p
        if element_rule not in N.ELEMENT_RULES:
            raise ValueError(f"unknown element rule {element_rule!r} (expected one of {sorted(N.ELEMENT_RULES)})")
        desc.element_rule = N.ELEMENT_RULES[element_rule]
        # per-node masks need the node count: a host-only analysis gives it
        probe = N.MeshDesc.from_buffer_copy(desc)
        probe.device = -1
        probe.leaf_max = leaf_max
        h = ctypes.c_void_p()
        N.check(L.pd_create_mesh(ctypes.byref(probe), ctypes.byref(h)), "pd_create_mesh")
        info = N.MeshInfo()
        L.pd_mesh_query(h, ctypes.byref(info))
        L.pd_mesh_destroy(h)
        n = info.n_nodes
        dir_arr, dir_p = _u8(dirichlet, n, "dirichlet")
        con_arr, con_p = _u8(contact, n, "contact")
        desc.dirichlet = dir_p
        desc.contact = con_p
        desc.leaf_max = leaf_max
        desc.device = -1 if device is None else int(device)
        self.device = device
        self.handle = ctypes.c_void_p()
        N.check(L.pd_create_mesh(ctypes.byref(desc), ctypes.byref(self.handle)), "pd_create_mesh")
        self._keep = [mask_arr, dir_arr, con_arr]
        self.info = self.query()
        self.n = self.info["n_nodes"]
        self.e = self.info["n_elems"]
        self.dx = dx
        self.h = None

    @classmethod
    def from_tet_mesh(cls, X, tets, density, dirichlet=None, contact=None, leaf_max=64,
                      device: Optional[int] = 0):
        """An unstructured tetrahedral mesh (pd_create_tet_mesh): X (n, 3) rest
        positions, tets (e, 4) vertex indices; nodes and tetrahedra keep the
        caller's order."""
        L = N.lib()
        self = cls.__new__(cls)
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
        tets = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
        n = X.shape[0]
        dir_arr, dir_p = _u8(dirichlet, n, "dirichlet")
        con_arr, con_p = _u8(contact, n, "contact")
        desc = N.TetMeshDesc()
        desc.n_nodes, desc.n_tets = n, tets.shape[0]
        desc.X = X.ctypes.data_as(N.c_double_p)
        desc.tets = tets.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        desc.density = density
        desc.dirichlet, desc.contact = dir_p, con_p
        desc.leaf_max = leaf_max
        desc.device = -1 if device is None else int(device)
        self._keep = [X, tets, dir_arr, con_arr]
        self.device = device
        self.handle = ctypes.c_void_p()
        N.check(L.pd_create_tet_mesh(ctypes.byref(desc), ctypes.byref(self.handle)), "pd_create_tet_mesh")
        self.info = self.query()
        self.n = self.info["n_nodes"]
        self.e = self.info["n_elems"]
        self.dx = None
        self.h = None
        return self

    @classmethod
    def from_tet_scene(cls, sc, leaf_max=64, device=0):
        return cls.from_tet_mesh(sc.X, sc.tets, sc.density, sc.dirichlet,
                                 getattr(sc, "contact", None) if sc.k_contact > 0 else None, leaf_max, device)

    @classmethod
    def from_scene(cls, sc, leaf_max=64, device=0):
        return cls(sc.nx, sc.ny, sc.nz, sc.dx, sc.density, tuple(sc.origin), sc.cell_mask, sc.dirichlet,
                   sc.contact if sc.k_contact > 0 else None, leaf_max, device,
                   getattr(sc, "element_rule", "hex8"))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            N.lib().pd_mesh_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self) -> dict:
        info = N.MeshInfo()
        N.check(N.lib().pd_mesh_query(self.handle, ctypes.byref(info)), "pd_mesh_query")
        return {k: getattr(info, k) for k, _ in info._fields_}

    def export(self, what: str) -> np.ndarray:
        L = N.lib()
        cnt = ctypes.c_int64()
        N.check(L.pd_mesh_export(self.handle, N.EXPORT[what], None, 0, ctypes.byref(cnt)), "pd_mesh_export")
        out = np.zeros(max(cnt.value, 1), dtype=np.int64)
        N.check(L.pd_mesh_export(self.handle, N.EXPORT[what], out.ctypes.data_as(N.c_i64_p), out.size,
                                 ctypes.byref(cnt)), "pd_mesh_export")
        return out[:cnt.value]

    # ------------------------------------------------------------------
    def factorize(self, w_corot=None, w_vol=None, w_muscle=None, fiber=None, h=0.01,
                  gravity=(0.0, 0.0, -9.81), k_contact=0.0, precision=N.PD_PREC_FP64, stream=None,
                  neohookean=False):
        """neohookean=True: Neo-Hookean material with mu = w_corot / 2, lambda = w_vol."""
        o = N.FactorOpts()
        o.h = h
        o.gravity = (ctypes.c_double * 3)(*gravity)
        o.k_contact = k_contact
        o.precision = precision
        o.neohookean = 1 if neohookean else 0
        self.h = h
        N.check(N.lib().pd_factorize(self.handle, _ptr(w_corot), _ptr(w_vol), _ptr(w_muscle), _ptr(fiber),
                                     ctypes.byref(o), _stream(stream)), "pd_factorize")

    def plan_checkpoints(self, T, mem_cap=0) -> int:
        """Checkpoint interval for a T-step rollout: 0 when every state fits in
        mem_cap bytes (0: four fifths of the free device memory), else the smallest
        K dividing T whose checkpoints and one recomputed segment fit."""
        K = ctypes.c_int32()
        N.check(N.lib().pd_plan_checkpoints(self.handle, int(T), int(mem_cap), ctypes.byref(K)),
                "pd_plan_checkpoints")
        return K.value

    def forward(self, x0, v0, T, f_ext=None, act=None, mu=0.0, opts=None, stream=None,
                allow_not_converged=False, mem_cap=0) -> Rollout:
        """With opts.checkpoint_every < 0 the interval is planned from mem_cap
        (pd_plan_checkpoints) and recorded in the returned Rollout.  f_ext is (n, 3),
        the same every step, or (T, n, 3), one external force per step."""
        opts = _with_fext_layout(opts or solver_opts(), f_ext, T, self.n)
        K = opts.checkpoint_every
        if K < 0:
            K = self.plan_checkpoints(T, mem_cap)
            opts = N.SolverOpts.from_buffer_copy(opts)
            opts.checkpoint_every = K
        S = T + 1 if K <= 0 else T // K + 1
        xs = torch.empty((S, self.n, 3), dtype=torch.float64, device=x0.device)
        vs = torch.empty_like(xs)
        st = N.Stats()
        status = N.lib().pd_forward(self.handle, _ptr(x0), _ptr(v0), _ptr(f_ext), _ptr(act), mu, T,
                                    ctypes.byref(opts), _ptr(xs), _ptr(vs), ctypes.byref(st), _stream(stream))
        N.check(status, "pd_forward", allow=(N.PD_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return Rollout(xs, vs, st.as_dict(), status, K)

    def backward(self, roll: Rollout, T, dL_dx, dL_dv=None, loss_all_steps=False, f_ext=None, act=None,
                 mu=0.0, opts=None, stream=None, want=("x0", "v0", "fext", "w_corot", "w_vol", "w_muscle",
                                                        "act", "mu"), allow_not_converged=False):
        opts = _with_fext_layout(opts or solver_opts(), f_ext, T, self.n)
        if opts.checkpoint_every < 0:   # planned by forward: the rollout carries it
            opts = N.SolverOpts.from_buffer_copy(opts)
            opts.checkpoint_every = roll.checkpoint_every
        dev = roll.x.device
        out = {}
        # the library reads loss_states blocks of (n, 3): check the caller's shapes here
        states = T + 1 if loss_all_steps else 1
        want_shape = (T + 1, self.n, 3) if loss_all_steps else (self.n, 3)
        for name, g in (("dL_dx", dL_dx), ("dL_dv", dL_dv)):
            if g is not None and tuple(g.shape) != want_shape:
                raise ValueError(f"{name}: expected shape {want_shape} (loss_all_steps={bool(loss_all_steps)}), "
                                 f"got {tuple(g.shape)}")
        K = opts.checkpoint_every
        S = T + 1 if K <= 0 else T // K + 1
        if tuple(roll.x.shape) != (S, self.n, 3) or tuple(roll.v.shape) != (S, self.n, 3):
            raise ValueError(f"rollout states: expected shape {(S, self.n, 3)} for checkpoint_every={K}, "
                             f"got {tuple(roll.x.shape)}")

        def alloc(name, shape):
            if name in want:
                out[name] = torch.zeros(shape, dtype=torch.float64, device=dev)
                return out[name]
            return None
        gx0 = alloc("x0", (self.n, 3))
        gv0 = alloc("v0", (self.n, 3))
        gf = alloc("fext", (T, self.n, 3) if opts.fext_per_step else (self.n, 3))
        gwc = alloc("w_corot", (self.e,))
        gwv = alloc("w_vol", (self.e,))
        gwm = alloc("w_muscle", (self.e,))
        ga = alloc("act", (T, self.e)) if act is not None else None
        gmu = alloc("mu", (1,))
        st = N.Stats()
        status = N.lib().pd_backward(self.handle, _ptr(roll.x), _ptr(roll.v), _ptr(f_ext), _ptr(act), mu, T,
                                     _ptr(dL_dx), _ptr(dL_dv), states, ctypes.byref(opts),
                                     _ptr(gx0), _ptr(gv0), _ptr(gf), _ptr(gwc), _ptr(gwv), _ptr(gwm), _ptr(ga),
                                     _ptr(gmu), ctypes.byref(st), _stream(stream))
        N.check(status, "pd_backward", allow=(N.PD_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        out["stats"] = st.as_dict()
        return out

    def local_step(self, x, act=None, precision=N.PD_PREC_FP64, stream=None):
        g = torch.empty((self.n, 3), dtype=torch.float64, device=x.device)
        e = torch.zeros((1,), dtype=torch.float64, device=x.device)
        N.check(N.lib().pd_local_step(self.handle, _ptr(x), _ptr(act), precision, _ptr(g), _ptr(e),
                                      _stream(stream)), "pd_local_step")
        return g, e

    def hessian_vector(self, x, v, act=None, precision=N.PD_PREC_FP64, stream=None):
        out = torch.empty((self.n, 3), dtype=torch.float64, device=x.device)
        N.check(N.lib().pd_hessian_vector(self.handle, _ptr(x), _ptr(act), _ptr(v), precision, _ptr(out),
                                          _stream(stream)), "pd_hessian_vector")
        return out

    # ---------------------------------------------------- complementarity contact
    def contact_prepare(self, candidates, stream=None):
        """L_A^-1 columns of the contact candidates (per kept node mask), after factorize."""
        arr, p = _u8(candidates, self.n, "candidates")
        N.check(N.lib().pd_contact_prepare(self.handle, p, _stream(stream)), "pd_contact_prepare")

    def contact_set(self, nodes, stream=None):
        """Fixes the contact set (kept node ids, each a candidate)."""
        arr = np.ascontiguousarray(np.asarray(nodes, dtype=np.int32).reshape(-1))
        N.check(N.lib().pd_contact_set(self.handle, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), arr.size,
                                       _stream(stream)), "pd_contact_set")
        self.contact_count = int(arr.size)

    def contact_step_set(self, t):
        """(nodes, ray) of step t of the last forward pass with complementarity
        contact: kept node ids in the order they joined and their target rule
        (True = ray intersection, False = dropped onto the ground)."""
        cnt = ctypes.c_int64(0)
        st = N.lib().pd_contact_step_set(self.handle, int(t), None, None, 0, ctypes.byref(cnt))
        if st != N.PD_OK and cnt.value == 0:
            N.check(st, "pd_contact_step_set")
        nodes = np.zeros(cnt.value, dtype=np.int32)
        rules = np.zeros(cnt.value, dtype=np.uint8)
        N.check(N.lib().pd_contact_step_set(self.handle, int(t), nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                            rules.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nodes.size,
                                            ctypes.byref(cnt)), "pd_contact_step_set")
        return nodes, rules.astype(bool)

    def solve_contact(self, b, x_star=None, precision=N.PD_PREC_FP64, stream=None):
        """x with x_C = x_star ((c,3), set order) and A_{C'C'} x_{C'} = b_{C'}."""
        out = torch.empty((self.n, 3), dtype=torch.float64, device=b.device)
        N.check(N.lib().pd_solve_A_contact(self.handle, _ptr(b), _ptr(x_star), _ptr(out), precision,
                                           _stream(stream)), "pd_solve_A_contact")
        return out

    def solve(self, b, precision=N.PD_PREC_FP64, stream=None):
        out = torch.empty((self.n, 3), dtype=torch.float64, device=b.device)
        N.check(N.lib().pd_solve_A(self.handle, _ptr(b), _ptr(out), precision, _stream(stream)), "pd_solve_A")
        return out


def scene_weights(sc, device="cuda"):
    """(w_corot, w_vol, w_muscle, fiber) device tensors for a workloads.Scene."""
    E = np.asarray(sc.youngs, dtype=np.float64)
    wc, wv = material_weights(E, sc.poisson)
    t = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64,
                                                         device=device)
    w_corot = t(wc) if sc.corotated else None
    w_vol = t(wv) if sc.volume else None
    w_m = t(E * np.asarray(sc.muscle, dtype=np.float64)) if sc.muscle is not None else None
    fib = t(sc.fiber) if sc.muscle is not None else None
    return w_corot, w_vol, w_m, fib


def _host(a, dtype, n=None, name=""):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype).reshape(-1))
    if n is not None and arr.size != n:
        raise ValueError(f"{name}: expected {n} entries, got {arr.size}")
    ptype = N.c_u8_p if dtype == np.uint8 else N.c_double_p
    return arr, arr.ctypes.data_as(ptype)


class PDServer:
    """Rollout-plus-gradient serving on one GPU (pd_serve_*): each request is a
    forward rollout, the loss sum(loss_w * x_T) and the backward pass to dL/dv0
    and dL/dact.  Requests are admitted continuously onto `max_slots` worker
    slots; see diffpd.h for the admission and caching rules."""

    def __init__(self, device=0, mem_budget=16 << 30, max_slots=4):
        self.handle = ctypes.c_void_p()
        N.check(N.lib().pd_serve_create(int(device), int(mem_budget), int(max_slots), ctypes.byref(self.handle)),
                "pd_serve_create")

    def submit_scene(self, sc, precision=N.PD_PREC_MIXED, opts=None, act=None, loss_w=None, T=None) -> int:
        """Submits a workloads.Scene; act / loss_w / T default to the scene's.
        Requests are hexahedral meshes (the request carries no element rule)."""
        if getattr(sc, "element_rule", "hex8") != "hex8":
            raise ValueError("serving requests are hexahedral meshes; got element rule "
                             f"{sc.element_rule!r}")
        E = np.asarray(sc.youngs, dtype=np.float64)
        wc, wv = material_weights(E, sc.poisson)
        e = E.size
        T = sc.T if T is None else T
        act = sc.act if act is None else act
        if act is not None:
            act = np.asarray(act, dtype=np.float64)[:T]
        loss_w = sc.loss_w if loss_w is None else loss_w
        r = N.Request()
        r.nx, r.ny, r.nz = sc.nx, sc.ny, sc.nz
        r.dx = sc.dx
        r.origin = (ctypes.c_double * 3)(*sc.origin)
        r.density = sc.density
        keep = []

        def put(field, a, dtype, n=None):
            arr, p = _host(a, dtype, n, field)
            keep.append(arr)
            setattr(r, field, p)
        n = sc.x0.shape[0]
        put("cell_mask_host", sc.cell_mask, np.uint8, sc.nx * sc.ny * sc.nz)
        put("dirichlet_host", sc.dirichlet, np.uint8, n)
        put("contact_host", sc.contact if sc.k_contact > 0 else None, np.uint8, n)
        put("w_corot_host", wc if sc.corotated else None, np.float64, e)
        put("w_vol_host", wv if sc.volume else None, np.float64, e)
        musc = sc.muscle is not None
        put("w_muscle_host", E * np.asarray(sc.muscle, dtype=np.float64) if musc else None, np.float64, e)
        put("fiber_host", sc.fiber if musc else None, np.float64, 3 * e)
        r.h = sc.h
        r.gravity = (ctypes.c_double * 3)(*sc.gravity)
        r.k_contact = sc.k_contact
        r.mu = sc.mu
        r.precision = precision
        r.T = T
        put("x0_host", sc.x0, np.float64, 3 * n)
        put("v0_host", sc.v0, np.float64, 3 * n)
        put("f_ext_host", sc.f_ext, np.float64, 3 * n)
        put("act_host", act, np.float64, T * e if act is not None else None)
        put("loss_w_host", loss_w, np.float64, 3 * n)
        r.opts = opts or solver_opts()
        t = ctypes.c_uint64()
        N.check(N.lib().pd_serve_submit(self.handle, ctypes.byref(r), ctypes.byref(t)), "pd_serve_submit")
        return t.value

    def poll(self, ticket: int):
        """None while pending; else a dict with the result (arrays copied)."""
        res = N.Result()
        st = N.lib().pd_serve_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(res))
        if st == N.PD_ERR_TIMEOUT:
            return None
        N.check(st, "pd_serve_poll")
        n, e, T = res.n_nodes, res.n_elems, res.T
        out = {k: getattr(res, k) for k in ("status", "loss", "queue_ms", "latency_ms", "fwd_iters", "bwd_iters",
                                            "slot", "mesh_cached", "factor_cached")}

        def arr(p, count, shape):
            if not p or res.status not in (N.PD_OK, N.PD_ERR_NOT_CONVERGED):
                return None
            return np.ctypeslib.as_array(p, shape=(count,)).reshape(shape).copy()
        out["x_final"] = arr(res.x_final_host, 3 * n, (n, 3))
        out["g_v0"] = arr(res.g_v0_host, 3 * n, (n, 3))
        out["g_act"] = arr(res.g_act_host, T * e, (T, e))
        return out

    def release(self, ticket: int):
        N.check(N.lib().pd_serve_release(self.handle, ctypes.c_uint64(ticket)), "pd_serve_release")

    def result(self, ticket: int):
        """Waits (host polling) for a ticket, returns its result and releases it."""
        import time
        while True:
            r = self.poll(ticket)
            if r is not None:
                self.release(ticket)
                return r
            time.sleep(0.0005)

    def drain(self):
        N.check(N.lib().pd_serve_drain(self.handle), "pd_serve_drain")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            N.lib().pd_serve_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
