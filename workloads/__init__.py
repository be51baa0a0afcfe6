"""Seeded synthetic scenes for the differentiable Projective Dynamics hot path.

This module only draws inputs: voxel-grid shapes, boundary masks, materials,
initial states, loss weights, tractions, actuation signals and request
streams.  It holds none of the method's arithmetic (no shape functions, no
mass lumping, no projections), so both the FP64 oracle and the CUDA path can
take their inputs from here without sharing any computation.

Grid conventions (both sides implement them independently):
  * grid node (i, j, k), 0 <= i <= nx, ..., has grid id (i*(ny+1)+j)*(nz+1)+k;
    i runs along the long axis x.
  * cell (ci, cj, ck) has cell id (ci*ny+cj)*nz+ck.
  * with a cell mask, kept cells keep their relative order and kept nodes
    (nodes touched by a kept cell) keep their relative order.
Per-node arrays below are indexed by kept node, per-element arrays by kept cell.

Random streams use NumPy PCG64 with seed = scene_index*1000 + stream_id.
"""
from .scenes import (  # noqa: F401
    Scene,
    grid_node_ids,
    kept_nodes,
    cantilever_c1,
    beam_c2,
    contact_cube_c3,
    quadruped,
    serving_stream_c4,
    beam_c5,
    small_beam,
    rolling_sphere,
    napkin,
    tet_beam,
    tet_ball,
    neohookean_beam,
    SCENES,
)
from .tetscenes import TetScene, unstructured_tet_ball, unstructured_tet_beam  # noqa: F401
