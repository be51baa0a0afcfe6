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
                checkpoint_every=0, check_every=4, profile=False, warm_start=False) -> N.SolverOpts:
    return N.SolverOpts(tol_fwd, tol_bwd, max_iter_fwd, max_iter_bwd, lbfgs_m, ls_max, checkpoint_every,
                        check_every, 1 if profile else 0, 1 if warm_start else 0)


@dataclass
class Rollout:
    x: torch.Tensor      # (S, n, 3)
    v: torch.Tensor
    stats: dict
    status: int


class PDMesh:
    """A voxel hex mesh resident on one GPU (pd_create_mesh ... pd_mesh_destroy)."""

    def __init__(self, nx, ny, nz, dx, density, origin=(0.0, 0.0, 0.0), cell_mask=None, dirichlet=None,
                 contact=None, leaf_max=64, device: Optional[int] = 0):
        L = N.lib()
        self._keep = []
        mask_arr, mask_p = _u8(cell_mask, nx * ny * nz, "cell_mask")
        desc = N.MeshDesc()
        desc.nx, desc.ny, desc.nz = nx, ny, nz
        desc.dx = dx
        desc.origin = (ctypes.c_double * 3)(*origin)
        desc.density = density
        desc.cell_mask = mask_p
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
    def from_scene(cls, sc, leaf_max=64, device=0):
        return cls(sc.nx, sc.ny, sc.nz, sc.dx, sc.density, tuple(sc.origin), sc.cell_mask, sc.dirichlet,
                   sc.contact if sc.k_contact > 0 else None, leaf_max, device)

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
                  gravity=(0.0, 0.0, -9.81), k_contact=0.0, precision=N.PD_PREC_FP64, stream=None):
        o = N.FactorOpts()
        o.h = h
        o.gravity = (ctypes.c_double * 3)(*gravity)
        o.k_contact = k_contact
        o.precision = precision
        self.h = h
        N.check(N.lib().pd_factorize(self.handle, _ptr(w_corot), _ptr(w_vol), _ptr(w_muscle), _ptr(fiber),
                                     ctypes.byref(o), _stream(stream)), "pd_factorize")

    def forward(self, x0, v0, T, f_ext=None, act=None, mu=0.0, opts=None, stream=None,
                allow_not_converged=False) -> Rollout:
        opts = opts or solver_opts()
        K = opts.checkpoint_every
        S = T + 1 if K <= 0 else T // K + 1
        xs = torch.empty((S, self.n, 3), dtype=torch.float64, device=x0.device)
        vs = torch.empty_like(xs)
        st = N.Stats()
        status = N.lib().pd_forward(self.handle, _ptr(x0), _ptr(v0), _ptr(f_ext), _ptr(act), mu, T,
                                    ctypes.byref(opts), _ptr(xs), _ptr(vs), ctypes.byref(st), _stream(stream))
        N.check(status, "pd_forward", allow=(N.PD_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return Rollout(xs, vs, st.as_dict(), status)

    def backward(self, roll: Rollout, T, dL_dx, dL_dv=None, loss_all_steps=False, f_ext=None, act=None,
                 mu=0.0, opts=None, stream=None, want=("x0", "v0", "fext", "w_corot", "w_vol", "w_muscle",
                                                        "act", "mu"), allow_not_converged=False):
        opts = opts or solver_opts()
        dev = roll.x.device
        out = {}

        def alloc(name, shape):
            if name in want:
                out[name] = torch.zeros(shape, dtype=torch.float64, device=dev)
                return out[name]
            return None
        gx0 = alloc("x0", (self.n, 3))
        gv0 = alloc("v0", (self.n, 3))
        gf = alloc("fext", (self.n, 3))
        gwc = alloc("w_corot", (self.e,))
        gwv = alloc("w_vol", (self.e,))
        gwm = alloc("w_muscle", (self.e,))
        ga = alloc("act", (T, self.e)) if act is not None else None
        gmu = alloc("mu", (1,))
        st = N.Stats()
        status = N.lib().pd_backward(self.handle, _ptr(roll.x), _ptr(roll.v), _ptr(f_ext), _ptr(act), mu, T,
                                     _ptr(dL_dx), _ptr(dL_dv), 1 if loss_all_steps else 0, ctypes.byref(opts),
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
