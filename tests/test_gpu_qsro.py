"""GPU parity of the qSRO path (Sec. IV-B, Eq. quadratic_local_SRO) against
the FP64 oracle, through the C ABI.

The sweep evaluates a trial's dE in FP32 from the species of a, b and the
sites within the model's shells of either, and from those sites' cached
own-species counts (the W terms).  Every trial's dE must lie within
DE_TOL_EV of the FP64 oracle and decide the same, except where the
acceptance threshold lies between the two values (the GPU then continues
from the oracle's state).  A sweep (its count cache carried through all its
mini-steps) must equal its traced mini-steps (the cache rebuilt from the
occupancy at each) bit for bit.  Energies and dE/dtheta come from exact
integer counts in FP64."""
import math

import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DE_TOL_EV = 1e-5  # FP32 dE vs FP64 (the bound the floating-point paths meet)


@pytest.fixture(scope="module")
def smc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08250_gb300 import build, smc as s
    build.build()
    s.lib()
    return s


def dev():
    return torch.device("cuda:0")


def models(smc, nsh, S, seed=7, zero_diag=False):
    """zero_diag: V^{pp} = 0, so that the linear sum over p' <= p is the
    paper's sum over p' < p exactly."""
    V, W, C = inputs.qsro_coeffs(seed, nsh, S)
    if zero_diag:
        for m in range(nsh):
            np.fill_diagonal(V[m], 0.0)
    return (smc.Model(smc.QSRO_F32, nsh, V, qsro_w=W, qsro_c=C),
            oracle.Model(oracle.QSRO, nsh, V, qsro_w=W, qsro_c=C))


def state(smc, dims, S, seed):
    """The oracle's start state, on the device (the oracle never reads a
    configuration the GPU produced)."""
    N = 2 * dims[0] * dims[1] * dims[2]
    lat = smc.Lattice(*dims, S)
    ref = oracle.init_lattice(oracle.Lattice(*dims, S), inputs.dirichlet_counts(N, S, seed), seed)
    return lat, torch.from_numpy(ref.copy()).to(dev()), ref


def accept_threshold(r, kT):
    """dE at which the test (r + 1/2) 2^-29 < exp(-dE / kT) flips."""
    return -kT * math.log((r + 0.5) * 2.0 ** -29)


def site_r(seed, replica, sweep, a):
    """r of site a: the low 29 bits of its Philox word (the oracle's RNG)."""
    w = oracle.philox4x32_10([a >> 2, replica, sweep & 0xFFFFFFFF, sweep >> 32],
                             [seed & 0xFFFFFFFF, seed >> 32])[a & 3]
    return int(w) & ((1 << 29) - 1)


@pytest.mark.parametrize("dims,nsh,kT,S,zero_diag", [((8, 8, 8), 2, 0.07, 5, False), ((12, 8, 16), 3, 0.05, 5, False),
                                                    ((8, 12, 8), 1, 0.1, 5, False), ((8, 8, 12), 3, 0.06, 8, False),
                                                    ((12, 12, 8), 2, 0.05, 2, False), ((8, 8, 8), 2, 0.07, 5, True),
                                                    ((12, 8, 8), 3, 0.05, 5, True)])
def test_lockstep_vs_oracle(smc, dims, nsh, kT, S, zero_diag):
    gm, om = models(smc, nsh, S, zero_diag=zero_diag)
    lat, occ, ref = state(smc, dims, S, 3)
    olat = oracle.Lattice(*dims, S)
    nA, _ = oracle.schedule(olat)
    nt = lat.nsites // nA
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    acc = torch.zeros(nt, dtype=torch.uint8, device=dev())
    worst, flips, n_acc = 0.0, 0, 0
    for t in range(2):
        for k in range(nA):
            smc.ministep_trace(lat, gm, occ, 11, t, k, kT, dE=dE, acc=acc)
            smc.check()
            want, wacc, a, b = oracle.ministep_trace(olat, om, ref, 11, t, k, kT)
            got, gacc = dE.cpu().numpy().astype(np.float64), acc.cpu().numpy().astype(bool)
            err = np.abs(got - want)
            worst = max(worst, float(err.max()))
            assert np.all(err <= DE_TOL_EV), (t, k, float(err.max()))
            bad = np.nonzero(gacc != wacc)[0]
            for i in bad:  # a flip needs the acceptance threshold between the two dE values
                thr = accept_threshold(site_r(11, 0, t, int(a[i])), kT)
                lo, hi = sorted((got[i], want[i]))
                slack = 1e-6 * kT  # the GPU evaluates exp in FP32
                assert lo - slack <= thr <= hi + slack, (t, k, i, got[i], want[i], thr)
            flips += len(bad)
            n_acc += int(gacc.sum())
            if len(bad):  # the GPU continues from the oracle's state
                occ.copy_(torch.from_numpy(ref.copy()).to(dev()))
            else:
                assert np.array_equal(occ.cpu().numpy(), ref), (t, k)
    assert n_acc > 0 and worst < DE_TOL_EV
    assert flips <= 2


@pytest.mark.parametrize("dims,nsh", [((8, 8, 8), 2), ((12, 8, 16), 3), ((32, 32, 32), 2), ((16, 8, 8), 1)])
def test_sweep_equals_trace(smc, dims, nsh):
    S = 5
    gm, _ = models(smc, nsh, S, seed=9)
    lat, occ, _ = state(smc, dims, S, 5)
    occ2 = occ.clone()
    kT = [0.06, 0.09]
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.sweep(lat, gm, occ, 4, 10, 2, kT, e_acc=e_acc, n_acc=n_acc)
    nA = 2 * 4 * 4 * 4
    nt = lat.nsites // nA
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    acc = torch.zeros(nt, dtype=torch.uint8, device=dev())
    n2 = 0
    for t in range(2):
        for k in range(nA):
            smc.ministep_trace(lat, gm, occ2, 4, 10 + t, k, kT[t], dE=dE, acc=acc)
            n2 += int(acc.sum().item())
    smc.check()
    assert torch.equal(occ, occ2)
    assert int(n_acc.item()) == n2


def test_energy_and_bookkeeping(smc):
    S, nsh, dims = 5, 3, (16, 8, 12)
    gm, om = models(smc, nsh, S)
    lat, occ, ref = state(smc, dims, S, 2)
    olat = oracle.Lattice(*dims, S)
    e0 = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.energy(lat, gm, occ, e0)
    smc.check()
    assert float(e0.item()) == pytest.approx(oracle.total_energy(olat, om, ref), rel=1e-12)
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.sweep(lat, gm, occ, 3, 0, 3, 0.08, e_acc=e_acc, n_acc=n_acc)
    e1 = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.energy(lat, gm, occ, e1)
    smc.check()
    host = occ.cpu().numpy()
    # accepted FP32 dE against the exact change: within DE_TOL_EV per trial as a random walk (6 sigma)
    n = int(n_acc.item())
    assert abs(float(e1.item()) - float(e0.item()) - float(e_acc.item())) <= 6 * math.sqrt(n) * DE_TOL_EV / math.sqrt(3)
    assert np.array_equal(np.bincount(host, minlength=S), inputs.dirichlet_counts(lat.nsites, S, 2))


@pytest.mark.parametrize("nsh", [1, 3])
def test_gradient_vs_oracle(smc, nsh):
    S, dims = 4, (8, 8, 8)
    gm, om = models(smc, nsh, S, seed=12)
    lat, occ, ref = state(smc, dims, S, 6)
    g = torch.zeros(smc.grad_size(lat, gm), dtype=torch.float32, device=dev())
    smc.energy_grad(lat, gm, occ, g)
    smc.check()
    want = oracle.energy_grad(oracle.Lattice(*dims, S), om, ref)
    assert g.numel() == want.size
    np.testing.assert_allclose(g.cpu().numpy().astype(np.float64), want, rtol=2 ** -23, atol=1e-6)


def test_unsupported_and_invalid(smc):
    S = 5
    gm, _ = models(smc, 2, S)
    lat, occ, _ = state(smc, (6, 8, 8), S, 1)  # 6 cells: one link cell along x
    with pytest.raises(smc.SMCError):
        smc.sweep(lat, gm, occ, 1, 0, 1, 0.1)
    lat2, occ2, _ = state(smc, (8, 8, 8), S, 1)
    with pytest.raises(smc.SMCError):
        smc.sweep_batched([lat2, lat2], gm, [occ2, occ2.clone()], 1, 0, 1, [0.1, 0.1])
    V, W, C = inputs.qsro_coeffs(1, 2, S)
    V[0, 0, 1] += 0.5  # not symmetric
    with pytest.raises(smc.SMCError):
        smc.sweep(lat2, smc.Model(smc.QSRO_F32, 2, V, qsro_w=W, qsro_c=C), occ2, 1, 0, 1, 0.1)


def test_full_size_256_sampled(smc):
    """256^3 cells, five species, 2-shell qSRO: one sweep of the GPU from the
    start state (composition conserved), then, on the oracle's start state,
    mini-step 0 of sweep 1 traced on the GPU and by the oracle: every trial
    within DE_TOL_EV."""
    S, nsh, dims = 5, 2, (256, 256, 256)
    gm, om = models(smc, nsh, S)
    lat, occ, ref = state(smc, dims, S, 1)
    counts = inputs.dirichlet_counts(lat.nsites, S, 1)
    smc.sweep(lat, gm, occ, 1, 0, 1, 0.07)
    smc.check()
    assert np.array_equal(np.bincount(occ.cpu().numpy(), minlength=S), counts)
    occ.copy_(torch.from_numpy(ref.copy()).to(dev()))
    nt = lat.nsites // 128
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    smc.ministep_trace(lat, gm, occ, 1, 1, 0, 0.07, dE=dE)
    smc.check()
    want, _, _, _ = oracle.ministep_trace(oracle.Lattice(*dims, S), om, ref, 1, 1, 0, 0.07)
    err = np.abs(dE.cpu().numpy().astype(np.float64) - want)
    assert float(err.max()) <= DE_TOL_EV
    assert np.array_equal(np.bincount(occ.cpu().numpy(), minlength=S), counts)
