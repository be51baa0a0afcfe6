"""Graph nested dissection of an unstructured tetrahedral mesh and its supernodal
structure (oracle; test infrastructure only).

The voxel meshes' ordering (oracle/structure.py) bisects grid boxes at node planes;
a mesh with its own node set has no planes, so the ordering here bisects by
coordinates and takes a vertex separator from the mesh graph (two free nodes are
adjacent when a tetrahedron holds both):

  dissect(S): a set S of free nodes with at most leaf_max members is a leaf (its
  nodes in increasing index order); otherwise order S by (position along the axis
  of S's largest extent -- ties x, y, z -- then node index), let L be the first
  floor(|S| / 2) nodes and R the rest, and let the separator C be the nodes of L
  adjacent to a node of R; then dissect(L \\ C), dissect(R), and append C (increasing
  index order) as one supernode when it is not empty.

The supernodes are the leaves and the non-empty separators; no node of one side is
adjacent to a node of the other, so L_A has no entry between them and they are
independent subtrees.  The row structure, parents and levels follow from the
adjacency exactly as for the voxel meshes (structure.supernodal_structure).
"""
from __future__ import annotations

import numpy as np

from .structure import supernodal_structure


def free_adjacency(tets, dirichlet):
    """Adjacency sets of the free nodes (free-node numbering, increasing node index)."""
    dirichlet = np.asarray(dirichlet, dtype=bool)
    free = np.flatnonzero(~dirichlet)
    fidx = -np.ones(dirichlet.size, dtype=np.int64)
    fidx[free] = np.arange(free.size)
    adj = [set() for _ in range(free.size)]
    for t in np.asarray(tets, dtype=np.int64):
        f = [int(fidx[a]) for a in t if fidx[a] >= 0]
        for a in f:
            adj[a].update(f)
    return free, adj


def nested_dissection(X, tets, dirichlet, leaf_max=64):
    """(perm, snode_first): perm[k] = free-node index of the k-th eliminated node."""
    free, adj = free_adjacency(tets, dirichlet)
    P = np.asarray(X, dtype=np.float64)[free]
    perm, firsts = [], []

    def rec(S):
        if S.size == 0:
            return
        if S.size <= leaf_max:
            firsts.append(len(perm))
            perm.extend(int(i) for i in np.sort(S))
            return
        ext = P[S].max(axis=0) - P[S].min(axis=0)
        axis = int(np.argmax(ext))   # first axis of the largest extent
        order = S[np.lexsort((S, P[S, axis]))]
        half = S.size // 2
        L, R = order[:half], order[half:]
        rset = set(int(i) for i in R)
        C = np.array(sorted(int(i) for i in L if adj[int(i)] & rset), dtype=np.int64)
        Lc = np.array(sorted(set(int(i) for i in L) - set(C.tolist())), dtype=np.int64)
        rec(Lc)
        rec(np.sort(R))
        if C.size:
            firsts.append(len(perm))
            perm.extend(int(i) for i in C)

    rec(np.arange(free.size, dtype=np.int64))
    firsts.append(len(perm))
    return np.array(perm, dtype=np.int64), np.array(firsts, dtype=np.int64)


def analyse(X, tets, dirichlet, leaf_max=64):
    """Ordering, adjacency in the permuted numbering and the supernodal structure."""
    perm, first = nested_dissection(X, tets, dirichlet, leaf_max)
    _, adj = free_adjacency(tets, dirichlet)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    padj = [sorted(int(inv[j]) for j in adj[int(perm[k])]) for k in range(perm.size)]
    st = supernodal_structure(first, padj)
    st["perm"] = perm
    st["snode_first"] = first
    st["adj"] = padj
    return st
