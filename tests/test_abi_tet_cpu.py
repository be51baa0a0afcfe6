"""The native host analysis of unstructured tetrahedral meshes (pd_create_tet_mesh
with device = -1, no GPU needed) reproduces the oracle's graph nested dissection
and supernodal structure (oracle/tetstructure.py) bit for bit, builds the node
incidence the definition gives, and rejects malformed meshes."""
import numpy as np
import pytest

from oracle import tetstructure
from workloads import unstructured_tet_beam


@pytest.fixture(scope="module")
def api():
    from paper_2101_05917_gb300 import build
    build.build()
    from paper_2101_05917_gb300 import api
    return api


CASES = [((6, 3, 3), 16, 11), ((8, 4, 4), 8, 12), ((8, 4, 4), 64, 13), ((5, 5, 5), 16, 14), ((12, 3, 2), 5, 15)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_tet_structures_bit_exact(api, case):
    (nx, ny, nz), leaf, index = CASES[case]
    sc = unstructured_tet_beam(nx, ny, nz, T=1, index=index)
    m = api.PDMesh.from_tet_scene(sc, leaf_max=leaf, device=None)
    st = tetstructure.analyse(sc.X, sc.tets, sc.dirichlet, leaf_max=leaf)
    for key in ("perm", "snode_first", "row_ptr", "rows", "parent", "level", "rel"):
        assert np.array_equal(m.export(key), st[key]), key
    assert np.array_equal(m.export("level_list"), np.concatenate(st["level_lists"]))
    # incidence: node -> entries e*8 + vertex, ascending
    n = sc.X.shape[0]
    entries = [[] for _ in range(n)]
    for e, t in enumerate(sc.tets):
        for a, v in enumerate(t):
            entries[v].append(8 * e + a)
    ptr = np.concatenate([[0], np.cumsum([len(x) for x in entries])])
    assert np.array_equal(m.export("inc_ptr"), ptr)
    assert np.array_equal(m.export("inc"), np.concatenate([sorted(x) for x in entries]))
    info = m.query()
    assert info["n_nodes"] == n and info["n_elems"] == sc.tets.shape[0]
    assert info["n_free"] == int((sc.dirichlet == 0).sum())
    m.close()


@pytest.mark.parametrize("jitter", [0.0, 0.05, 0.45])
@pytest.mark.parametrize("leaf", [3, 8])
def test_tet_ordering_bit_exact_under_coordinate_ties(api, jitter, leaf):
    """jitter 0 puts every node on the lattice (whole planes of equal coordinates,
    so the ordering's ties are broken by node index throughout)."""
    for index in (3, 4):
        sc = unstructured_tet_beam(5, 4, 3, T=1, index=index, jitter=jitter)
        m = api.PDMesh.from_tet_scene(sc, leaf_max=leaf, device=None)
        st = tetstructure.analyse(sc.X, sc.tets, sc.dirichlet, leaf_max=leaf)
        for key in ("perm", "snode_first", "row_ptr", "rows", "parent", "level", "rel"):
            assert np.array_equal(m.export(key), st[key]), (key, index)
        m.close()


def test_tet_mesh_rejects_malformed_input(api):
    from paper_2101_05917_gb300 import _native as N
    sc = unstructured_tet_beam(3, 2, 2, T=1)

    def status(X, tets, dirichlet=None):
        with pytest.raises(N.PDError) as err:
            api.PDMesh.from_tet_mesh(X, tets, 1e3, dirichlet, device=None)
        return err.value.status
    bad = sc.tets.copy()
    bad[0, 1] = sc.X.shape[0]                       # vertex out of range
    assert status(sc.X, bad) == N.PD_ERR_INVALID_ARG
    bad = sc.tets.copy()
    bad[1, 2] = bad[1, 0]                           # repeated vertex
    assert status(sc.X, bad) == N.PD_ERR_INVALID_ARG
    X = sc.X.copy()
    t = sc.tets[2]
    X[t[3]] = X[t[0]] + 0.5 * (X[t[1]] - X[t[0]])  # vertex 3 on edge 0-1: zero volume
    assert status(X, sc.tets) == N.PD_ERR_INVALID_ARG
    X = sc.X.copy()
    p0, p1, p2 = X[t[0]], X[t[1]], X[t[2]]
    nrm = np.cross(p1 - p0, p2 - p0)
    nrm /= np.linalg.norm(nrm)
    X[t[3]] = (p0 + p1 + p2) / 3 + 1e-15 * nrm      # a sliver of volume ~1e-15 of its edge cubed
    assert status(X, sc.tets) == N.PD_ERR_INVALID_ARG
    X = np.vstack([sc.X, [[1.0, 1.0, 1.0]]])        # a node in no tetrahedron
    assert status(X, sc.tets) == N.PD_ERR_INVALID_ARG
    assert status(sc.X, sc.tets, np.ones(sc.X.shape[0])) == N.PD_ERR_INVALID_ARG   # nothing free
    # either orientation is accepted and gives the same structure
    flipped = sc.tets[:, [0, 2, 1, 3]]
    a = api.PDMesh.from_tet_mesh(sc.X, sc.tets, 1e3, sc.dirichlet, device=None)
    b = api.PDMesh.from_tet_mesh(sc.X, flipped, 1e3, sc.dirichlet, device=None)
    for key in ("perm", "rows", "parent"):
        assert np.array_equal(a.export(key), b.export(key))


@pytest.mark.parametrize("leaf", [8, 64])
def test_tet_ball_without_fixed_nodes(api, leaf):
    """A free-floating contact ball (no fixed node, a contact mask): ordering and
    structure as the oracle's, every node free."""
    from workloads import unstructured_tet_ball
    sc = unstructured_tet_ball(T=1)
    m = api.PDMesh.from_tet_scene(sc, leaf_max=leaf, device=None)
    st = tetstructure.analyse(sc.X, sc.tets, sc.dirichlet, leaf_max=leaf)
    for key in ("perm", "snode_first", "row_ptr", "rows", "parent", "level", "rel"):
        assert np.array_equal(m.export(key), st[key]), key
    assert m.query()["n_free"] == sc.X.shape[0]
    m.close()
