"""Pins of the oracle's RNG, geometry and link-cell schedule (CPU only)."""
import numpy as np
import pytest

import oracle
from tests import helpers


def test_philox_known_answers():
    for ctr, key, want in helpers.read_kat():
        assert [int(x) for x in oracle.philox4x32_10(ctr, key)] == want


def test_shell_vectors_match_distance_enumeration():
    for m in (1, 2, 3):
        got = sorted(tuple(int(c) for c in v) for v in oracle.shell_vectors(m))
        assert got == helpers.shell_vectors_bruteforce(m)
        assert len(got) == helpers.SHELL_Z[m]
    # shell 1 order: lexicographic with - before + (partner index = w >> 29)
    s1 = oracle.shell_vectors(1)
    assert [tuple(v) for v in s1] == sorted(tuple(v) for v in s1)
    assert tuple(s1[0]) == (-1, -1, -1) and tuple(s1[7]) == (1, 1, 1)


@pytest.mark.parametrize("dims", [(6, 6, 6), (4, 6, 8), (2, 2, 2), (3, 5, 2)])
def test_neighbor_matches_bruteforce(dims):
    lat = oracle.Lattice(*dims, 2)
    for m in (1, 2, 3):
        tab = helpers.neighbor_table(*dims, m)
        vecs = helpers.shell_vectors_bruteforce(m)
        for s in range(lat.nsites):
            for t, v in enumerate(vecs):
                assert oracle.neighbor(lat, s, v) == tab[s, t]


def test_neighbor_by_minimum_image_distance():
    """On a 6^3 box (no aliasing up to shell 3) the shells are exactly the
    sites at the three smallest periodic distances."""
    nx = ny = nz = 6
    p = helpers.positions(nx, ny, nz)
    L = 2 * np.array([nx, ny, nz])
    d = p[:, None, :] - p[None, :, :]
    d = (d + L // 2) % L - L // 2
    d2 = (d * d).sum(-1)
    lat = oracle.Lattice(nx, ny, nz, 2)
    for m in (1, 2, 3):
        for s in (0, 7, 215, 216, 300, lat.nsites - 1):
            want = set(np.nonzero(d2[s] == helpers.SHELL_D2[m])[0].tolist())
            got = {oracle.neighbor(lat, s, v) for v in oracle.shell_vectors(m)}
            assert got == want and len(want) == helpers.SHELL_Z[m]


def test_neighbor_inverse():
    lat = oracle.Lattice(8, 12, 4, 3)
    rng = np.random.default_rng(0)
    for s in rng.integers(0, lat.nsites, 200):
        for m in (1, 2, 3):
            for v in oracle.shell_vectors(m):
                t = oracle.neighbor(lat, s, v)
                assert oracle.neighbor(lat, t, -v) == s


@pytest.mark.parametrize("dims,L", [((8, 8, 8), (4, 4, 4)), ((12, 8, 16), (4, 4, 4)),
                                    ((2, 2, 2), (2, 2, 2)), ((6, 8, 4), (6, 4, 4)),
                                    ((10, 8, 8), (10, 4, 4))])
def test_schedule(dims, L):
    lat = oracle.Lattice(*dims, 2)
    nA, got = oracle.schedule(lat)
    assert got == L and nA == 2 * L[0] * L[1] * L[2]


def _read_write_sets(dims, reach):
    """Write set {a, b} and read set (Omega plus the sites its local energies
    read) of every possible trial, over all 8 partners."""
    tabs = [helpers.neighbor_table(*dims, m) for m in range(1, reach + 1)]
    nb = np.concatenate(tabs, axis=1)  # [N, z]
    s1 = helpers.neighbor_table(*dims, 1)
    return nb, s1


@pytest.mark.parametrize("dims", [(8, 8, 8), (12, 8, 16), (8, 12, 8)])
@pytest.mark.parametrize("reach", [2, 3])
def test_trials_of_a_ministep_are_independent(dims, reach):
    """No trial of a mini-step writes a site that another trial of the same
    mini-step reads (Sec. II-A: concurrent trials in distinct link cells).
    This is what makes the serial in-place oracle equal to Algorithm 1."""
    lat = oracle.Lattice(*dims, 2)
    nA, L = oracle.schedule(lat)
    nb, s1 = _read_write_sets(dims, reach)
    N = lat.nsites
    nx, ny, nz = dims
    for k in range(nA):
        dx = k % L[0]
        r = k // L[0]
        dy = r % L[1]
        r //= L[1]
        dz = r % L[2]
        sub = r // L[2]
        xs = np.arange(dx, nx, L[0])
        ys = np.arange(dy, ny, L[1])
        zs = np.arange(dz, nz, L[2])
        zz, yy, xx = np.meshgrid(zs, ys, xs, indexing="ij")
        a = (((sub * nz + zz) * ny + yy) * nx + xx).reshape(-1)
        owner_w = -np.ones(N, dtype=np.int64)
        # write sets over all partners: a and its 8 first neighbours
        for t, site in enumerate(a):
            for w in [site] + list(s1[site]):
                assert owner_w[w] in (-1, t)
                owner_w[w] = t
        # read sets: Omega (a, b, their neighbours) and Omega's neighbours
        for t, site in enumerate(a):
            om = set([site]) | set(s1[site].tolist())
            om |= set(nb[list(om)].reshape(-1).tolist())
            rd = om | set(nb[list(om)].reshape(-1).tolist())
            others = owner_w[list(rd)]
            assert np.all((others == -1) | (others == t))
