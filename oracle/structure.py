"""Index structures of the global step, re-derived from their definitions
(oracle; test infrastructure only).

The global step solves with the constant SPD matrix A (Eqn 19) whose
Cholesky factor is computed once (Sec. 3, "the Cholesky factorization of A
can be precomputed, after which each global step requires back-substitution
only").  Because G_c acts identically on the x, y and z coordinates, A is
I_3 (x) L_A for one scalar matrix L_A over the free nodes, whose pattern is the
27-point node adjacency of the hex mesh.  The paper gives no ordering or
supernode scheme (it calls Eigen); the definitions below are this
implementation's own and must be reproduced bit for bit by the native code:

  incidence   rows = kept nodes ascending; entries e*8+a (element e, corner a)
              of the cells touching the node, ascending.
  ordering    nested dissection over grid boxes of free nodes: a box with more
              than leaf_max free nodes is split along its longest axis (ties:
              x before y before z) at the node plane mid = floor((lo+hi)/2);
              the left part [lo, mid-1] is numbered first, then the right part
              [mid+1, hi], then the free nodes of the plane in natural (grid id)
              order.  A box with 1..leaf_max free nodes is a leaf numbered in
              natural order.
  supernodes  every leaf and every non-empty separator plane is one supernode
              (a contiguous range of columns).
  structure   rows(s) = cols(s) + {r >= first(s): L_A[r, c] != 0, c in s}
              + below(t) for every child t, sorted; below(s) = rows beyond
              last(s); parent(s) = supernode holding min(below(s)), or -1.
  levels      level(s) = 0 without children, else 1 + max over children;
              level lists are sorted by supernode id.
  rel         for each supernode with a parent p: the position of each row of
              below(s) inside rows(p).
"""
from __future__ import annotations

import numpy as np


def kept_mesh(nx, ny, nz, cell_mask):
    """(elems as grid ids (e,8), kept grid ids (n,))."""
    cells = []
    for ci in range(nx):
        for cj in range(ny):
            for ck in range(nz):
                cid = (ci * ny + cj) * nz + ck
                if cell_mask is not None and not cell_mask[cid]:
                    continue
                cells.append([((ci + ((a >> 2) & 1)) * (ny + 1) + (cj + ((a >> 1) & 1))) * (nz + 1)
                              + (ck + (a & 1)) for a in range(8)])
    cells = np.array(cells, dtype=np.int64).reshape(-1, 8)
    return cells, np.unique(cells.ravel())


def incidence(nx, ny, nz, cell_mask):
    """Node -> (element, corner) CSR: (row_ptr (n+1,), entries (8e,))."""
    cells, grid = kept_mesh(nx, ny, nz, cell_mask)
    index = {g: i for i, g in enumerate(grid.tolist())}
    lists = [[] for _ in range(grid.size)]
    for e in range(cells.shape[0]):
        for a in range(8):
            lists[index[int(cells[e, a])]].append(e * 8 + a)
    row_ptr = np.zeros(grid.size + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(l) for l in lists])
    entries = np.array([v for l in lists for v in sorted(l)], dtype=np.int64)
    return row_ptr, entries


def nested_dissection(nx, ny, nz, cell_mask, dirichlet, leaf_max=64):
    """Returns (perm, snode_first): perm[new] = free-node index (free nodes in
    kept order), snode_first[s] = first column of supernode s (plus n_free)."""
    cells, grid = kept_mesh(nx, ny, nz, cell_mask)
    dirichlet = np.asarray(dirichlet, dtype=bool)
    free_grid = grid[~dirichlet]
    free_index = {int(g): i for i, g in enumerate(free_grid.tolist())}
    k = free_grid % (nz + 1)
    j = (free_grid // (nz + 1)) % (ny + 1)
    i = free_grid // ((nz + 1) * (ny + 1))
    ijk = np.stack([i, j, k], axis=1)
    perm = []
    firsts = []

    def nodes_in(lo, hi):
        m = np.all((ijk >= lo) & (ijk <= hi), axis=1)
        return free_grid[m]                      # ascending grid id

    def rec(lo, hi):
        ids = nodes_in(lo, hi)
        if ids.size == 0:
            return
        if ids.size <= leaf_max:
            firsts.append(len(perm))
            perm.extend(free_index[int(g)] for g in ids)
            return
        ext = hi - lo + 1
        d = int(np.argmax(ext))
        mid = (lo[d] + hi[d]) // 2
        lhi = hi.copy(); lhi[d] = mid - 1
        rlo = lo.copy(); rlo[d] = mid + 1
        slo = lo.copy(); slo[d] = mid
        shi = hi.copy(); shi[d] = mid
        rec(lo.copy(), lhi)
        rec(rlo, hi.copy())
        sep = nodes_in(slo, shi)
        if sep.size:
            firsts.append(len(perm))
            perm.extend(free_index[int(g)] for g in sep)

    rec(np.array([0, 0, 0]), np.array([nx, ny, nz]))
    firsts.append(len(perm))
    return np.array(perm, dtype=np.int64), np.array(firsts, dtype=np.int64)


def permuted_adjacency(nx, ny, nz, cell_mask, dirichlet, perm):
    """Adjacency lists of L_A in the permuted numbering (each sorted, incl. self)."""
    cells, grid = kept_mesh(nx, ny, nz, cell_mask)
    dirichlet = np.asarray(dirichlet, dtype=bool)
    kept_index = {int(g): i for i, g in enumerate(grid.tolist())}
    free_of_kept = -np.ones(grid.size, dtype=np.int64)
    free_of_kept[~dirichlet] = np.arange(np.count_nonzero(~dirichlet))
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    adj = [set() for _ in range(perm.size)]
    for e in range(cells.shape[0]):
        cols = [free_of_kept[kept_index[int(g)]] for g in cells[e]]
        cols = [int(inv[c]) for c in cols if c >= 0]
        for a in cols:
            adj[a].update(cols)
    return [sorted(s) for s in adj]


def supernodal_structure(snode_first, adj):
    """Row structure, parent, levels, level lists and relative indices."""
    ns = snode_first.size - 1
    nf = int(snode_first[-1])
    owner = np.empty(nf, dtype=np.int64)
    for s in range(ns):
        owner[snode_first[s]:snode_first[s + 1]] = s
    rows = []
    parent = -np.ones(ns, dtype=np.int64)
    children = [[] for _ in range(ns)]
    for s in range(ns):
        f, l = int(snode_first[s]), int(snode_first[s + 1])
        r = set(range(f, l))
        for c in range(f, l):
            r.update(x for x in adj[c] if x >= f)
        for t in children[s]:
            r.update(x for x in rows[t] if x >= int(snode_first[t + 1]))
        rs = np.array(sorted(r), dtype=np.int64)
        rows.append(rs)
        below = rs[rs >= l]
        if below.size:
            p = int(owner[below[0]])
            parent[s] = p
            children[p].append(s)
    level = np.zeros(ns, dtype=np.int64)
    for s in range(ns):
        if children[s]:
            level[s] = 1 + max(level[t] for t in children[s])
    n_levels = int(level.max()) + 1 if ns else 0
    level_lists = [np.flatnonzero(level == L) for L in range(n_levels)]
    rel = []
    for s in range(ns):
        p = int(parent[s])
        below = rows[s][rows[s] >= int(snode_first[s + 1])]
        if p < 0:
            rel.append(np.zeros(0, dtype=np.int64))
        else:
            rel.append(np.searchsorted(rows[p], below).astype(np.int64))
    row_ptr = np.zeros(ns + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([r.size for r in rows])
    return {
        "row_ptr": row_ptr,
        "rows": np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64),
        "parent": parent,
        "level": level,
        "level_lists": level_lists,
        "rel": np.concatenate(rel) if rel else np.zeros(0, dtype=np.int64),
    }


def analyse(nx, ny, nz, cell_mask, dirichlet, leaf_max=64):
    """All index structures of one mesh."""
    perm, first = nested_dissection(nx, ny, nz, cell_mask, dirichlet, leaf_max)
    adj = permuted_adjacency(nx, ny, nz, cell_mask, dirichlet, perm)
    st = supernodal_structure(first, adj)
    st["perm"] = perm
    st["snode_first"] = first
    st["adj"] = adj
    rp, ent = incidence(nx, ny, nz, cell_mask)
    st["inc_ptr"] = rp
    st["inc"] = ent
    return st
