"""Interaction lists (§2.2 step 3): the tensor-core contraction never stores
its lists; each CTA enumerates the offsets of its target parity itself.  This
test restates that enumeration (the order in which the producer, the MMA
issuer and the epilogue walk the offsets, and how a source cell is addressed
from its parity block and coarse shift) and checks it, entry by entry and in
order, against the list the oracle's downward pass iterates over, for every
target parity at levels 1-7, open and periodic."""
import numpy as np
import pytest

import oracle


def kernel_offsets(bx, by, bz):
    """The contraction's offset walk for target parity (bx, by, bz): x fastest,
    then y, then z over [-2 - b, 3 - b] per axis, skipping |o|_inf <= 1; each
    offset's source parity and coarse shift."""
    out = []
    ox, oy, oz = -2 - bx - 1, -2 - by, -2 - bz
    while True:
        while True:  # one step of the walk, repeated while the offset is adjacent
            ox += 1
            if ox > 3 - bx:
                ox = -2 - bx
                oy += 1
                if oy > 3 - by:
                    oy = -2 - by
                    oz += 1
                    if oz > 3 - bz:
                        return out
            if not (-1 <= ox <= 1 and -1 <= oy <= 1 and -1 <= oz <= 1):
                break
        sx, sy, sz = bx + ox, by + oy, bz + oz
        spar = (sx & 1) | ((sy & 1) << 1) | ((sz & 1) << 2)
        out.append((((oz + 3) * 7 + (oy + 3)) * 7 + (ox + 3), spar, sx >> 1, sy >> 1, sz >> 1))


def kernel_list(l, periodic, cx, cy, cz):
    """The sources the contraction reads for target (cx, cy, cz) of level l: the
    coarse cell (X + dX, Y + dY, Z + dZ) of parity block spar, i.e. the cell
    2 (X + dX) + (spar & 1), ...; open: a source outside the box is a zero halo
    cell (it adds nothing and is not in the list); periodic: the wrapped image."""
    S = 1 << l
    X, Y, Z = cx >> 1, cy >> 1, cz >> 1
    src, oi = [], []
    for o, spar, dX, dY, dZ in kernel_offsets(cx & 1, cy & 1, cz & 1):
        sx = 2 * (X + dX) + (spar & 1)
        sy = 2 * (Y + dY) + ((spar >> 1) & 1)
        sz = 2 * (Z + dZ) + (spar >> 2)
        if periodic:
            sx, sy, sz = sx % S, sy % S, sz % S
        elif not (0 <= sx < S and 0 <= sy < S and 0 <= sz < S):
            continue
        src.append((sz * S + sy) * S + sx)
        oi.append(o)
    return np.array(src, np.int64), np.array(oi, np.int32)


def _cells(l, rng):
    """Every cell of small levels; corners, faces and seeded interior cells of
    every parity for the others."""
    S = 1 << l
    if S <= 8:
        return [(x, y, z) for z in range(S) for y in range(S) for x in range(S)]
    edge = [0, 1, 2, 3, S // 2 - 1, S // 2, S - 4, S - 3, S - 2, S - 1]
    cells = [(x, y, z) for z in edge for y in edge[::3] for x in edge]
    cells += [tuple(int(v) for v in rng.integers(0, S, 3)) for _ in range(64)]
    return cells


def test_offset_walk_covers_the_list_definition():
    """189 offsets per parity, |o|_inf >= 2, parents within one cell of each
    other; 316 = 7^3 - 3^3 distinct offsets over the eight parities."""
    allo = set()
    for par in range(8):
        b = (par & 1, (par >> 1) & 1, par >> 2)
        offs = kernel_offsets(*b)
        assert len(offs) == 189 == len(set(o[0] for o in offs))
        for o, *_ in offs:
            ox, oy, oz = o % 7 - 3, (o // 7) % 7 - 3, o // 49 - 3
            assert max(abs(ox), abs(oy), abs(oz)) >= 2
            for a, oa in zip(b, (ox, oy, oz)):
                assert ((a + oa) >> 1) in (-1, 0, 1)
        allo |= set(o[0] for o in offs)
    assert len(allo) == 316


@pytest.mark.parametrize("periodic", [False, True])
def test_kernel_lists_match_the_oracle(periodic):
    rng = np.random.default_rng(7)
    for l in range(1 if periodic else 2, 8):
        for (cx, cy, cz) in _cells(l, rng):
            s_o, o_o = oracle.interaction_list(l, periodic, cx, cy, cz)
            s_k, o_k = kernel_list(l, periodic, cx, cy, cz)
            np.testing.assert_array_equal(s_k, s_o, err_msg=str((l, periodic, cx, cy, cz)))
            np.testing.assert_array_equal(o_k, o_o, err_msg=str((l, periodic, cx, cy, cz)))
            if periodic or min(cx, cy, cz) >= 4 and max(cx, cy, cz) < (1 << l) - 4:
                assert len(s_o) == 189
