"""Host model of the mixed paths' U cube layout (no GPU).

The tensor-core contractions store each group tensor as its term of W in W's
own index order (C0[a][b][c] = U0, C1[b][a][c] = U1, C2[b][c][a] = U2), in 8^3
cubes whose three group terms lie side by side; inside a cube, element
(x, y, z) sits at ucube_off(x, y, z) in C0 and C1 and at ucube_off(x, z, y) in
C2 (tcorr_internal.cuh).  The epilogue copies the 6 KB of a cube position and
reads W = C0 + C1 + C2 element by element.  These tests restate the swizzle,
the store formula of store_u_cubes (tc_common.cuh) and the epilogue's reads,
and check the properties the kernels rely on:
  - the offsets are a bijection of the 512 cells;
  - the six ways the epilogue walks a cube (a warp holds 4 consecutive values
    of one index and all 8 of another, the third fixed) touch 32 distinct
    shared-memory banks;
  - a warp's store (2 values of b x 16 of c at fixed a) fills 4 whole
    32-byte sectors in every group;
  - stores and reads agree: W[x][y][z] = U0[x][y][z] + U1[y][x][z] + U2[z][x][y]
    (the grouped form of eq. symm_operator, tcorr_internal.cuh), ragged v
    included.
"""
import itertools

import numpy as np
import pytest


def ucube_off(x, y, z):
    return (x << 6) | ((y ^ (x & 3)) << 3) | (z ^ y ^ (x & 4))


def c2_off(x, y, z):
    return ucube_off(x, z, y)


@pytest.mark.parametrize("off", [ucube_off, c2_off])
def test_offsets_are_a_bijection(off):
    cells = sorted(off(x, y, z) for x in range(8) for y in range(8) for z in range(8))
    assert cells == list(range(512))


@pytest.mark.parametrize("off", [ucube_off, c2_off])
def test_every_epilogue_walk_is_bank_conflict_free(off):
    # thread (la, lb, lc): lb = 4 beta .. 4 beta + 3 and lc = 0..7 within a warp, la fixed;
    # the six orderings abc, acb, bac, bca, cab, cba of the element orbit
    walks = [lambda a, b, c: (a, b, c), lambda a, b, c: (a, c, b), lambda a, b, c: (b, a, c),
             lambda a, b, c: (b, c, a), lambda a, b, c: (c, a, b), lambda a, b, c: (c, b, a)]
    for la, beta, walk in itertools.product(range(8), range(2), walks):
        banks = {off(*walk(la, 4 * beta + lb, lc)) % 32 for lb in range(4) for lc in range(8)}
        assert len(banks) == 32


def store_cells(g, a7, lb_pair, lc16):
    """Cube cells (cube index offset, in-cube offset) a warp's store writes for
    group g at a & 7 = a7: b & 7 in lb_pair, c = 0..15 across two c cubes."""
    cells = []
    for lb in lb_pair:
        for c in range(lc16):
            cz, lc = c >> 3, c & 7
            if g == 0:
                cells.append((cz, ucube_off(a7, lb, lc)))
            elif g == 1:
                cells.append((cz, ucube_off(lb, a7, lc)))
            else:  # C2[b][c][a] with its y index innermost
                cells.append((cz, c2_off(lb, lc, a7)))
    return cells


@pytest.mark.parametrize("g", [0, 1, 2])
def test_a_warps_store_fills_whole_sectors(g):
    for a7, lb0 in itertools.product(range(8), range(0, 8, 2)):
        cells = store_cells(g, a7, (lb0, lb0 + 1), 16)
        sectors = {(cz, off // 8) for cz, off in cells}
        assert len(sectors) == 4 and len(cells) == 32  # 4 sectors of 8 floats, all written


@pytest.mark.parametrize("v", [8, 13, 21])
def test_stores_and_epilogue_reads_agree(v):
    rng = np.random.default_rng(v)
    nb = (v + 7) // 8
    U = [rng.standard_normal((v, v, v)) for _ in range(3)]  # U^g[a][b][c]
    task = np.full(3 * nb ** 3 * 512, np.nan)
    # store_u_cubes: thread (b, c), a = a0 + j, a0 a multiple of 8
    for g in range(3):
        for b, c in itertools.product(range(v), range(v)):
            B, C, lb, lc = b >> 3, c >> 3, b & 7, c & 7
            for a in range(v):
                A, q = a >> 3, a & 7
                if g == 0:
                    cell = ((A * nb + B) * nb + C) * 3 * 512 + (ucube_off(0, lb, lc) ^ ucube_off(q, 0, 0))
                elif g == 1:
                    cell = (((B * nb + A) * nb + C) * 3 + 1) * 512 + (ucube_off(lb, 0, lc) ^ ucube_off(0, q, 0))
                else:
                    cell = (((B * nb + C) * nb + A) * 3 + 2) * 512 + (ucube_off(lb, 0, lc) ^ ucube_off(0, q, 0))
                task[cell] = U[g][a, b, c]
    # the epilogue: the 6 KB at cube (X, Y, Z), W = C0 + C1 + C2
    for x, y, z in itertools.product(range(v), repeat=3):
        base = (((x >> 3) * nb + (y >> 3)) * nb + (z >> 3)) * 3 * 512
        lx, ly, lz = x & 7, y & 7, z & 7
        w = task[base + ucube_off(lx, ly, lz)] + task[base + 512 + ucube_off(lx, ly, lz)] + \
            task[base + 1024 + c2_off(lx, ly, lz)]
        assert w == pytest.approx(U[0][x, y, z] + U[1][y, x, z] + U[2][z, x, y], rel=1e-14, abs=1e-14)
