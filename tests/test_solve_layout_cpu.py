"""The triangular solve's tile schedule and its streamed FP32 layout, from the host
analysis (no GPU).  Each chunk of a tile reaches shared memory by one bulk copy,
which must start on a 16-byte boundary and move a multiple of 16 bytes, at most the
32 KB stage: a copy that breaks these rules is an illegal instruction on the GPU,
so they are checked here for every chunk of every test mesh (voxel meshes, and
unstructured tetrahedral meshes up to the bench's, whose graph-ordered supernodes
have irregular sizes), together with the
chunks lying back to back.  The schedule itself must equal a re-derivation from
its definition: per supernode (nc columns, nr rows), forward tiles are row blocks
of R rows (R = 256 for nc <= 32, 128 for nc <= 64, else 64) over the columns
[0, cend) their rows need (a row block inside the triangular L11^-1 block only up
to its last row), in chunks of 256/R column groups of 32 columns; backward tiles
are column blocks of BC columns (the narrowest of 8/16/32/64 covering nc, 64 at
most) over the rows from their first column down, in chunks of min(8192/BC, 256)
rows; a level whose blocks number fewer than 608 has them cut into runs of at
most max(1, chunks of the level / 608) consecutive chunks (a tile each);
forward tiles by ascending tree level, backward tiles by descending level,
supernodes in level-list order.  Streamed copy per chunk: forward [group][column <
kmax_g][row < rv] with kmax_g = clamp(L - 32 g, 0, 32) for a chunk of L columns
(the groups filled in order), backward [column < bcv][row < rn]; each padded to
16 bytes."""
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
    LEVEL_TILES = 608

    def kc_of(blocks):
        total = sum(b[3] for b in blocks)
        most = max([b[3] for b in blocks] + [1])
        if len(blocks) >= LEVEL_TILES:
            return most
        return max(1, min(most, total // LEVEL_TILES))

    def split(blocks, kc, full_ld, out):
        for s, kind, a, nch, full, last, lld in blocks:
            nt = (nch + kc - 1) // kc
            for k in range(nt):
                c0 = k * kc
                n = min(kc, nch - c0)
                has_last = c0 + n == nch
                ld = lld if has_last else full_ld(kind)
                lastsz = last if has_last else full
                out.append((s, kind, a, c0, n, full, lastsz, ld, nt))

    for L in range(len(lp) - 1):
        fb, bb = [], []
        for s in ll[lp[L]:lp[L + 1]]:
            nc, nr = int(sf[s + 1] - sf[s]), int(rp[s + 1] - rp[s])
            R = 256 if nc <= 32 else (128 if nc <= 64 else 64)
            G = 256 // R
            CW = 32 * G
            for r0 in range(0, nr, R):
                rv = min(R, nr - r0)
                rmax = r0 + rv - 1
                cend = min(nc, rmax + 1) if rmax < nc else nc
                nch = (cend + CW - 1) // CW
                lld = cend - (nch - 1) * CW          # columns of the block's last chunk
                fb.append((s, KINDS_F[R], r0, nch, G * 32 * rv, lld * rv, lld))
            BC = 64 if nc > 32 else (32 if nc > 16 else (16 if nc > 8 else 8))
            BR = min(8192 // BC, 256)
            for c0 in range(0, nc, BC):
                rows = nr - c0
                nch = (rows + BR - 1) // BR
                lld = rows - (nch - 1) * BR
                bcv = min(BC, nc - c0)
                bb.append((s, KINDS_B[BC], c0, nch, bcv * BR, bcv * lld, lld))
        split(fb, kc_of(fb), lambda kind: 32 * {0: 1, 1: 2, 2: 4}[kind], fwd)
        lev_b = []
        bc_of = {3: 64, 4: 32, 5: 16, 6: 8}
        split(bb, kc_of(bb), lambda kind: min(8192 // bc_of[kind], 256), lev_b)
        bwd.append(lev_b)
    tiles = fwd + [t for lev in reversed(bwd) for t in lev]
    out, off = [], 0
    for s, kind, a, c0, n, full, last, ld, nt in tiles:
        lpad = (last + 3) // 4 * 4
        out.append((s, kind, a, c0, n, off, 4 * full, 4 * lpad, ld, nt))
        off += full * (n - 1) + lpad
    return np.array(out, dtype=np.int64).reshape(-1, 10)


CASES = [(cantilever_c1, 64), (cantilever_c1, 8), (lambda: quadruped(9, T=1), 64),
         (lambda: small_beam(5, 3, 4, T=1), 5), (lambda: contact_cube_c3(N=6, T=1), 32),
         (lambda: tet_ball(T=1), 16), (lambda: beam_c2(T=1), 64)]


# unstructured tetrahedral meshes: graph-ordered supernodes of irregular sizes
TET_CASES = [((6, 3, 3), 16), ((8, 4, 4), 8), ((16, 8, 8), 64), ((24, 12, 12), 64), ((48, 24, 24), 64)]


@pytest.mark.parametrize("case", range(len(CASES) + len(TET_CASES)))
def test_solve_tiles_match_definition_and_copy_rules(native, case):
    from paper_2101_05917_gb300 import api
    if case < len(CASES):
        make, leaf = CASES[case]
        m = api.PDMesh.from_scene(make(), leaf_max=leaf, device=None)
    else:
        from workloads import unstructured_tet_beam
        (nx, ny, nz), leaf = TET_CASES[case - len(CASES)]
        sc = unstructured_tet_beam(nx, ny, nz, T=1, index=21, E=1e6)
        m = api.PDMesh.from_tet_scene(sc, leaf_max=leaf, device=None)
    got = m.export("solve_tiles").reshape(-1, 10)
    want = _derive(m)
    assert np.array_equal(got, want)
    nch, soff, cbytes, lbytes = got[:, 4], got[:, 5], got[:, 6], got[:, 7]
    assert np.all(nch >= 1)
    assert np.all(soff % 4 == 0)                          # 16-byte aligned starts (floats)
    for b in (cbytes, lbytes):
        assert np.all(b % 16 == 0) and np.all(b > 0) and np.all(b <= 32768)
    # chunks back to back: every chunk but a tile's last has cbytes, the last lbytes
    ends = soff + (nch - 1) * (cbytes // 4) + lbytes // 4
    assert np.array_equal(soff[1:], ends[:-1])
    m.close()
