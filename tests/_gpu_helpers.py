"""Shared helpers for the GPU parity tests (inputs from workloads/, reference
values from oracle/, computation through the C ABI)."""
import numpy as np
import torch

from paper_2101_05917_gb300 import api
from paper_2101_05917_gb300 import _native as N

DEV = torch.device("cuda:0")


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def make_mesh(sc, precision=N.PD_PREC_FP64, leaf_max=64):
    mesh = api.PDMesh.from_scene(sc, leaf_max=leaf_max, device=0)
    wc, wv, wm, fib = api.scene_weights(sc, DEV)
    mesh.factorize(wc, wv, wm, fib, h=sc.h, gravity=tuple(sc.gravity), k_contact=sc.k_contact,
                   precision=precision, neohookean=getattr(sc, "neohookean", False))
    return mesh


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def deformed(sc, scale=0.02, seed=0, rotate=True):
    """Rest positions under a random rotation plus a random displacement field."""
    rng = np.random.default_rng(seed)
    x = sc.x0.copy()
    if rotate:
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        if np.linalg.det(Q) < 0:
            Q[:, 0] *= -1
        x = x @ Q.T
    return x + scale * sc.dx * rng.standard_normal(x.shape)
