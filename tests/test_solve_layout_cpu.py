"""The triangular solve's tile schedule and its streamed FP32 layout, from the host
analysis (no GPU).  Each tile's panel values reach shared memory by one bulk copy,
which must start on a 16-byte boundary and move a multiple of 16 bytes, at most the
48 KB tile stage: a copy that breaks these rules is an illegal instruction on the
GPU, so they are checked here for every tile of every test mesh, together with the
tiles lying back to back.  The schedule itself must equal a re-derivation from its
definition: per supernode (nc columns, nr rows), forward tiles of R rows (R = 256
for nc <= 48, 128 for nc <= 96, else 64) by 256/R column groups of 48, where a row
block inside the triangular L11^-1 block only takes columns up to its last row;
backward tiles of BC columns (the narrowest of 8/16/32/64 covering nc, 64 at most)
by min(12288/BC, 1024) rows, starting at the row block that holds the tile's first
column; forward tiles by ascending tree level, backward tiles by descending level,
supernodes in level-list order.  Streamed copy per tile: forward [group][column <
kmax][row < rv] with kmax the columns of the tile's last row inside its first
group, backward [column < bcv][row < rn]; each padded to 16 bytes."""
import numpy as np
import pytest

from workloads import cantilever_c1, contact_cube_c3, quadruped, small_beam, tet_ball, beam_c2

@pytest.fixture(scope="module")
def native():
    from paper_2101_05917_gb300 import build
    build.build()
    from paper_2101_05917_gb300 import _native
    return _native


KINDS_F = {256: 0, 128: 1, 64: 2}
KINDS_B = {64: 3, 32: 4, 16: 5, 8: 6}


def _derive(m):
    sf = m.export("snode_first")
    rp = m.export("row_ptr")
    ll = m.export("level_list")
    lp = m.export("level_ptr")
    fwd, bwd = [], []
    for L in range(len(lp) - 1):
        lev_b = []
        for s in ll[lp[L]:lp[L + 1]]:
            nc, nr = int(sf[s + 1] - sf[s]), int(rp[s + 1] - rp[s])
            R = 256 if nc <= 48 else (128 if nc <= 96 else 64)
            G = 256 // R
            for r0 in range(0, nr, R):
                cmax = r0 + R if r0 + R <= nc else nc
                rv = min(R, nr - r0)
                rmax = r0 + rv - 1
                cend = min(nc, rmax + 1) if rmax < nc else nc
                for c0 in range(0, cmax, 48 * G):
                    kmax = max(0, min(48, cend - c0))
                    fwd.append((s, KINDS_F[R], r0, c0, G * kmax * rv, kmax))
            BC = 64 if nc > 32 else (32 if nc > 16 else (16 if nc > 8 else 8))
            BR = min(12288 // BC, 1024)
            for c0 in range(0, nc, BC):
                for r0 in range((c0 // BR) * BR, nr, BR):
                    rn = min(BR, nr - r0)
                    lev_b.append((s, KINDS_B[BC], c0, r0, min(BC, nc - c0) * rn, rn))
        bwd.append(lev_b)
    tiles = fwd + [t for lev in reversed(bwd) for t in lev]
    out, off = [], 0
    for s, kind, a, b, elems, ld in tiles:
        padded = (elems + 3) // 4 * 4
        out.append((s, kind, a, b, off, 4 * padded, ld))
        off += padded
    return np.array(out, dtype=np.int64).reshape(-1, 7)


CASES = [(cantilever_c1, 64), (cantilever_c1, 8), (lambda: quadruped(9, T=1), 64),
         (lambda: small_beam(5, 3, 4, T=1), 5), (lambda: contact_cube_c3(N=6, T=1), 32),
         (lambda: tet_ball(T=1), 16), (lambda: beam_c2(T=1), 64)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_solve_tiles_match_definition_and_copy_rules(native, case):
    from paper_2101_05917_gb300 import api
    make, leaf = CASES[case]
    sc = make()
    m = api.PDMesh.from_scene(sc, leaf_max=leaf, device=None)
    got = m.export("solve_tiles").reshape(-1, 7)
    want = _derive(m)
    assert np.array_equal(got, want)
    soff, sbytes = got[:, 4], got[:, 5]
    assert np.all(soff % 4 == 0)                          # 16-byte aligned starts (floats)
    assert np.all(sbytes % 16 == 0) and np.all(sbytes > 0) and np.all(sbytes <= 49152)
    assert np.array_equal(soff[1:], soff[:-1] + sbytes[:-1] // 4)   # back to back
    m.close()
