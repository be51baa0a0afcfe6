"""Pins for the index-structure oracle: the nested-dissection permutation is a
permutation whose separators separate, the supernodal row structure contains
the exact fill of the Cholesky factor (brute-force dense elimination), the
supernodal tree is consistent, and the incidence CSR inverts the element list."""
import numpy as np
import pytest

from oracle import structure
from oracle.model import Model
from workloads import cantilever_c1, small_beam, quadruped


def _cases():
    c1 = cantilever_c1(T=1)
    q = quadruped(8, T=1)
    sb = small_beam(5, 3, 4, T=1)
    return [(c1, 64), (c1, 8), (q, 16), (sb, 5)]


@pytest.mark.parametrize("case", range(4))
def test_structure_contains_exact_fill(case):
    sc, leaf = _cases()[case]
    st = structure.analyse(sc.nx, sc.ny, sc.nz, sc.cell_mask, sc.dirichlet, leaf_max=leaf)
    perm = st["perm"]
    nf = perm.size
    assert np.array_equal(np.sort(perm), np.arange(nf))
    m = Model(sc)
    A = m.A_matrix()
    xd = m.free_nodes * 3
    LA = A[xd][:, xd].toarray()[np.ix_(perm, perm)]
    # adjacency lists agree with the numeric pattern of L_A
    for i in range(nf):
        assert np.array_equal(np.flatnonzero(LA[i]), st["adj"][i])
    L = np.linalg.cholesky(LA)
    first = st["snode_first"]
    owner = np.repeat(np.arange(first.size - 1), np.diff(first))
    allowed = np.zeros((nf, nf), dtype=bool)
    for s in range(first.size - 1):
        rows = st["rows"][st["row_ptr"][s]:st["row_ptr"][s + 1]]
        allowed[np.ix_(rows, np.arange(first[s], first[s + 1]))] = True
    fill = np.abs(L) > 1e-13 * np.abs(L).max()
    assert not np.any(fill & ~allowed)
    # the factor is exactly dense on each supernode's diagonal block
    for s in range(first.size - 1):
        blk = L[first[s]:first[s + 1], first[s]:first[s + 1]]
        assert np.all(np.diag(blk) > 0)
    # parents hold higher ids, levels increase towards the root, rel is consistent
    par = st["parent"]
    for s in range(first.size - 1):
        if par[s] >= 0:
            assert par[s] > s and st["level"][par[s]] > st["level"][s]
    rel = st["rel"]
    off = 0
    for s in range(first.size - 1):
        rows = st["rows"][st["row_ptr"][s]:st["row_ptr"][s + 1]]
        below = rows[rows >= first[s + 1]]
        if par[s] >= 0:
            prow = st["rows"][st["row_ptr"][par[s]]:st["row_ptr"][par[s] + 1]]
            assert np.array_equal(prow[rel[off:off + below.size]], below)
            off += below.size
        else:
            assert below.size == 0
    assert off == rel.size
    # level lists partition the supernodes
    assert sorted(np.concatenate(st["level_lists"]).tolist()) == list(range(first.size - 1))


def test_separators_separate():
    sc = small_beam(6, 5, 4, T=1)
    st = structure.analyse(sc.nx, sc.ny, sc.nz, sc.cell_mask, sc.dirichlet, leaf_max=6)
    first = st["snode_first"]
    par = st["parent"]
    owner = np.repeat(np.arange(first.size - 1), np.diff(first))

    def ancestors(s):
        out = {s}
        while par[s] >= 0:
            s = int(par[s])
            out.add(s)
        return out
    # a column only couples (in L_A) to its own supernode or its ancestors / descendants
    for i, nb in enumerate(st["adj"]):
        for j in nb:
            a, b = owner[i], owner[j]
            assert a in ancestors(b) or b in ancestors(a)


def test_incidence_inverts_element_list():
    sc = quadruped(8, T=1)
    rp, ent = structure.incidence(sc.nx, sc.ny, sc.nz, sc.cell_mask)
    m = Model(sc)
    for node in range(m.mesh.n):
        got = ent[rp[node]:rp[node + 1]]
        e, a = got // 8, got % 8
        assert np.all(m.mesh.elems[e, a] == node)
        assert np.all(np.diff(got) > 0)
    assert rp[-1] == 8 * m.mesh.e
