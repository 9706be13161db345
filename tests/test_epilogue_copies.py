"""Host model of the mixed epilogue's copy plan (no GPU).

Per block orbit (A <= B <= C) the producer warps of epilogue_f32_kernel
(epilogue.cu) fill a stage with: one 6 KB bulk copy of the three group
terms of each distinct cube slot, and 4-row TMA gathers of the blocked FP32
ovov copy (27 8x8 sub-blocks), of the t1 rows (9) and of the float-float
virtual energies (3 blocks).  The stage's mbarrier is armed with the byte
count the producers expect.  These tests restate that plan for every orbit
of several block counts and check what the kernel relies on:
  - the expected bytes equal the bytes the copies write (else the stage's
    wait would only end by its time limit);
  - every source lies inside its buffer and every gather row inside its
    tensor map;
  - the copies land inside the stage, without overlap, on the offsets the
    compute warps read (stage layout: cube[6][3][512] floats, ov[27][64] +
    one pad row, t1[9][8] + 3 pad rows, ev[3][8] float2 + one pad row);
  - the slots that repeat an earlier slot's block triple are not copied, and
    the compute warps' slot map points each slot at a copied slot with the
    same triple.
"""
import itertools

import pytest

STAGE_CUBE, STAGE_OV, STAGE_T1, STAGE_EV = 0, 36864, 36864 + 28 * 256, 36864 + 28 * 256 + 12 * 32
STAGE_BYTES = STAGE_EV + 4 * 64


def perm_pos(s, d):
    """Block position (0 = A, 1 = B, 2 = C) on axis d of slot s (abc, acb, bac, bca, cab, cba)."""
    p0 = s >> 1
    lo = 1 if p0 == 0 else 0
    hi = 1 if p0 == 2 else 2
    if d == 0:
        return p0
    return lo if (d == 1) == ((s & 1) == 0) else hi


def plan(o, nb, task, orbit):
    """The copies of one orbit: (kind, dst, bytes, source check) and the expected bytes."""
    ti, tj, tk = task
    ob = orbit
    triples = [tuple(ob[perm_pos(s, d)] for d in range(3)) for s in range(6)]
    smap = [next(t for t in range(s + 1) if triples[t] == triples[s]) for s in range(6)]
    loaded = [s for s in range(6) if smap[s] == s]
    copies = []
    for s in loaded:  # bulk copy of the three group terms of cube (X, Y, Z)
        X, Y, Z = triples[s]
        src = ((X * nb + Y) * nb + Z) * 3 * 512 * 4
        copies.append(("u", STAGE_CUBE + s * 6144, 6144, src, 3 * nb ** 3 * 512 * 4))
    copies.append(("ev", STAGE_EV, 4 * 64, max(ob[0], ob[1], ob[2]), nb))  # rows ob0, ob1, ob2, ob0
    for k in range(7):
        rows = []
        for u in range(4):
            q = min(4 * k + u, 26)
            sl, ba, bc = q // 9, (q // 3) % 3, q % 3
            first = tj if sl == 0 else ti
            second = tj if sl == 2 else tk
            rows.append(((first * o + second) * nb + ob[ba]) * nb + ob[bc])
        copies.append(("ov", STAGE_OV + k * 1024, 1024, max(rows), o * o * nb * nb))
    for k in range(3):
        rows = []
        for u in range(4):
            q = min(4 * k + u, 8)
            oc, b = q // 3, q % 3
            rows.append((ti, tj, tk)[oc] * nb + ob[b])
        copies.append(("t1", STAGE_T1 + k * 128, 128, max(rows), o * nb))
    expected = len(loaded) * 3 * 2048 + 4 * 64 + (7 * 4 * 256 + 3 * 4 * 32)
    return copies, expected, smap, triples


def orbits(nb):
    return [(a, b, c) for a in range(nb) for b in range(a, nb) for c in range(b, nb)]


@pytest.mark.parametrize("o,nb", [(2, 1), (3, 2), (4, 3), (5, 7)])
def test_copy_plan_is_consistent(o, nb):
    tasks = [(i, j, k) for i in range(o) for j in range(i, o) for k in range(j, o) if not i == j == k]
    for task, orbit in itertools.product(tasks[:6], orbits(nb)):
        copies, expected, smap, triples = plan(o, nb, task, orbit)
        assert sum(c[2] for c in copies) == expected
        spans = sorted((c[1], c[1] + c[2]) for c in copies)
        assert spans[0][0] >= 0 and spans[-1][1] <= STAGE_BYTES
        assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:])), "copies overlap"
        for kind, dst, nbytes, src, limit in copies:
            if kind == "u":
                assert src + nbytes <= limit            # inside the task's U block
            else:
                assert 0 <= src < limit                 # the largest row inside its map
            assert dst % (16 if kind == "u" else 128) == 0
        for s in range(6):
            assert smap[s] <= s and triples[smap[s]] == triples[s]
        assert (len(set(triples)) == 6) == (orbit[0] < orbit[1] < orbit[2])


def test_stage_layout_matches_the_kernel():
    # ov[27][64] + 1 pad row, t1[9][8] + 3 pad rows, ev[3][8] float2 + 1 pad row
    assert STAGE_OV == 6 * 3 * 512 * 4
    assert STAGE_T1 == STAGE_OV + 27 * 256 + 256
    assert STAGE_EV == STAGE_T1 + 9 * 32 + 3 * 32
    assert STAGE_BYTES == 44672 and STAGE_BYTES % 128 == 0
    # two CTAs per SM: two stages, alignment slack and 8576 bytes of static shared memory each
    assert 2 * (2 * STAGE_BYTES + 128 + 8576) <= 228 * 1024
