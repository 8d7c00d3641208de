"""The overlap rules the sweep kernels rely on, checked exhaustively on the
link-cell schedule (CPU, no oracle needed: a property of the mini-step order).

With four-cell link cells, the four mini-steps that share (sub, dy, dz) form a
group g = (sub * 4 + dz) * 4 + dy, and the trials of one x-row of link cells
(a column (cy, cz)) in a group read whole lattice rows (sublattice, y, z):
the trial sublattice's rows y0-1..y0+1 x z0-1..z0+1 and the partner
sublattice's rows y0+s_off-1..y0+s_off+2 (same in z; without the four corners
for two shells), with y0 = 4 cy + dy, z0 = 4 cz + dz, s_off = -1 on
sublattice 0 and 0 on 1.  They write the trial row (y0, z0) and the partner
rows y0+s_off+{0,1} x z0+s_off+{0,1}.  The kernels stage and write back
whole rows, so the rules must hold row by row:

* in one group, distinct columns touch disjoint rows (they run at once);
* a group with dy >= 1 shares no row with the previous group of any of the 8
  neighbouring columns -- no read of a row the other writes, in either order,
  and no row written by both -- so it may run while its neighbours still run
  that previous group (the kernels' lag of 2 groups); groups with dy = 0 wait
  for the previous group of their neighbours (lag 1).
"""
import pytest


def column_rows(cy, cz, g, ny, nz, nshells):
    dy, dz, sub = g & 3, (g >> 2) & 3, g >> 4
    soff = -1 if sub == 0 else 0
    y0, z0 = 4 * cy + dy, 4 * cz + dz
    reads = {(sub, (y0 + a) % ny, (z0 + b) % nz) for a in (-1, 0, 1) for b in (-1, 0, 1)}
    for sy in range(4):
        for sz in range(4):
            if nshells < 3 and sy in (0, 3) and sz in (0, 3):
                continue
            reads.add((1 - sub, (y0 + soff - 1 + sy) % ny, (z0 + soff - 1 + sz) % nz))
    writes = {(sub, y0 % ny, z0 % nz)}
    writes |= {(1 - sub, (y0 + soff + a) % ny, (z0 + soff + b) % nz) for a in (0, 1) for b in (0, 1)}
    assert writes <= reads
    return reads, writes


@pytest.mark.parametrize("ny,nz", [(8, 8), (12, 16), (16, 16), (24, 20), (32, 28)])
@pytest.mark.parametrize("nshells", [2, 3])
def test_group_overlap_rules(ny, nz, nshells):
    NLy, NLz = ny // 4, nz // 4
    rows = {(cy, cz, g): column_rows(cy, cz, g, ny, nz, nshells)
            for cy in range(NLy) for cz in range(NLz) for g in range(32)}
    for g in range(32):
        gp = (g - 1) % 32
        for cy in range(NLy):
            for cz in range(NLz):
                R, W = rows[(cy, cz, g)]
                for ey in (-1, 0, 1):
                    for ez in (-1, 0, 1):
                        c2 = ((cy + ey) % NLy, (cz + ez) % NLz)
                        if c2 == (cy, cz):
                            continue
                        R3, _ = rows[(*c2, g)]
                        assert not (R & R3), ("same group", g, (cy, cz), c2)
                        if g & 3:
                            R2, W2 = rows[(*c2, gp)]
                            assert not (W2 & R) and not (W & R2), ("lag 2", g, (cy, cz), c2)


def test_dy0_groups_do_need_the_previous_group():
    """The rule is tight: a dy = 0 group does read a row its neighbour
    writes in the previous group (so its lag of 1 is needed)."""
    ny = nz = 16
    found = False
    for g in range(0, 32, 4):
        gp = (g - 1) % 32
        R, _ = column_rows(1, 1, g, ny, nz, 2)
        for ey in (-1, 0, 1):
            for ez in (-1, 0, 1):
                if (ey, ez) != (0, 0):
                    _, W2 = column_rows(1 + ey, 1 + ez, gp, ny, nz, 2)
                    found |= bool(W2 & R)
    assert found
