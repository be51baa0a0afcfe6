"""Writes the stored oracle results used by the GPU parity tests.

Only oracle/ and workloads/ are called: every stored value comes from the FP64
CPU oracle (Newton forward, direct adjoint), never from the CUDA path.
Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import adjoint, newton  # noqa: E402
from oracle.model import Model  # noqa: E402
from workloads import cantilever_c1  # noqa: E402


def c1():
    sc = cantilever_c1()
    model = Model(sc)
    xs, vs, infos = newton.rollout(model, sc.x0, sc.v0, sc.f_ext)
    loss, gx = adjoint.final_position_loss(model, xs, sc.loss_w)
    g = adjoint.backward(model, xs, vs, gx)
    gE, gnu = adjoint.material_gradients(model, g)
    np.savez_compressed(os.path.join(HERE, "c1_cantilever_oracle.npz"), xs=xs, vs=vs, loss=loss,
                        g_v0=g["g_v0"], g_x0=g["g_x0"], g_wc=g["g_wc"], g_E=gE, g_nu=gnu,
                        newton_iters=np.array([i["iters"] for i in infos]))


if __name__ == "__main__":
    c1()
    print("written")
