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


@pytest.mark.parametrize("ny,nz", [(8, 8), (12, 16), (16, 16), (24, 20)])
def test_paired_groups_touch_disjoint_rows(ny, nz):
    """The paired streaming kernel runs groups (dy, dy + 1), dy = 0 or 2, of a
    column back to back once the neighbours have finished the previous pair,
    while the neighbours run the same pair in any interleaving: the rows one
    column reads or writes in the pair and the rows a neighbouring column
    writes in it must not meet (and no row is written by both)."""
    NLy, NLz = ny // 4, nz // 4
    for g in range(0, 32, 2):
        for cy in range(NLy):
            for cz in range(NLz):
                R = set().union(*(column_rows(cy, cz, g + h, ny, nz, 2)[0] for h in (0, 1)))
                W = set().union(*(column_rows(cy, cz, g + h, ny, nz, 2)[1] for h in (0, 1)))
                for ey in (-1, 0, 1):
                    for ez in (-1, 0, 1):
                        c2 = ((cy + ey) % NLy, (cz + ez) % NLz)
                        if c2 == (cy, cz):
                            continue
                        W2 = set().union(*(column_rows(*c2, g + h, ny, nz, 2)[1] for h in (0, 1)))
                        assert not (R & W2) and not (W & W2), ("pair", g, (cy, cz), c2)


def test_pairs_need_the_previous_pair():
    """A pair does read rows its neighbours wrote in their previous pair, so
    the paired kernel's wait for it is needed."""
    ny = nz = 16
    found = False
    for g in range(0, 32, 2):
        R = set().union(*(column_rows(1, 1, g + h, ny, nz, 2)[0] for h in (0, 1)))
        for ey in (-1, 0, 1):
            for ez in (-1, 0, 1):
                if (ey, ez) != (0, 0):
                    W2 = set().union(*(column_rows(1 + ey, 1 + ez, (g - 2 + h) % 32, ny, nz, 2)[1] for h in (0, 1)))
                    found |= bool(W2 & R)
    assert found


def exchange_hazards(ny, nz, by, bz, gps, ahead):
    """Rows the resident kernel's exchange would overwrite while its block
    still uses them.  Steps of gps groups; for step n the exchange fetches the
    versions of rows another block wrote last (at step w < n) and this block
    has not read since w, while the compute warps may still run steps
    n - ahead .. n - 1.  A hazard: such a row read or written by this block
    at one of those steps before w (after w it would have been fetched
    then).  Counted over a whole sweep for blocks of by x bz columns."""
    NLy, NLz = ny // 4, nz // 4
    NBy = (NLy + by - 1) // by
    S = 32 // gps

    def blk(cy, cz):
        return (cz // bz) * NBy + cy // by

    reads = [dict() for _ in range(S)]
    writes = [dict() for _ in range(S)]
    writer = [dict() for _ in range(S)]
    for st in range(S):
        for h in range(gps):
            for cy in range(NLy):
                for cz in range(NLz):
                    R, W = column_rows(cy, cz, st * gps + h, ny, nz, 2)
                    b = blk(cy, cz)
                    reads[st].setdefault(b, set()).update(R)
                    writes[st].setdefault(b, set()).update(W)
                    for r in W:
                        writer[st][r] = b
    bad = 0
    for b in range(NBy * ((NLz + bz - 1) // bz)):
        for n in range(S, 2 * S):
            for r in reads[n % S].get(b, ()):
                w = next((n - d for d in range(1, S + 1) if r in writer[(n - d) % S]), None)
                if w is None or writer[w % S][r] == b:
                    continue
                if any(r in reads[h % S].get(b, ()) for h in range(w + 1, n)):
                    continue
                for h in range(n - ahead, min(n, w)):
                    bad += r in reads[h % S].get(b, ()) or r in writes[h % S].get(b, ())
    return bad


@pytest.mark.parametrize("ny,nz,by,bz", [(32, 32, 2, 4), (24, 24, 2, 2), (16, 24, 1, 2)])
def test_resident_exchange_never_overwrites_a_row_in_use(ny, nz, by, bz):
    """The resident kernel fetches single groups up to two groups ahead of the
    compute warps: no fetched row is still in use (exchange_hazards).  The
    check is not vacuous: steps of two groups fetched two steps ahead would
    overwrite rows in use."""
    assert exchange_hazards(ny, nz, by, bz, 1, 2) == 0
    if (ny, nz) == (32, 32):
        assert exchange_hazards(ny, nz, by, bz, 2, 2) > 0
        assert exchange_hazards(ny, nz, by, bz, 2, 1) == 0
