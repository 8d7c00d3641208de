"""Statistical check of the FP32 GPU chain against the FP64 oracle on the
anneal workload's model (five species at equal counts, FP32 pair
coefficients over two shells drawn N(0, 20 meV), the 128^3 job's coefficient
seed), on a box the oracle finishes in seconds.

Each side runs 48 independent chains (different Philox seeds on the two
sides): a linear anneal from 3000 K to 300 K over 150 sweeps, then 100 sweeps
at 300 K.  Per chain, the final-window means (last 100 sweeps) of the energy
and of the like-pair Warren-Cowley parameters alpha_m^{pp} of shells 1 and 2
are taken; the GPU and oracle means over chains must agree within 3 standard
errors of their difference (the spread across chains, which also holds the
annealing path's seed-to-seed variation: the final energy of one chain
spreads over about 3.5 eV, so 48 chains per side resolve a shift of about
2 eV).  The oracle chains run in a pool of spawned processes.  On the same
seed the GPU chain repeats the oracle's to the last digit unless an FP32 dE
falls across an acceptance threshold, which is why independent seeds are used
here: the comparison is of distributions, not of trajectories."""
import math
import multiprocessing as mp

import numpy as np
import pytest

from paper_2604_08250_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS, S, NSH = (12, 12, 12), 5, 2
N_ANNEAL, N_HOLD, WINDOW = 150, 100, 100
GPU_SEEDS = list(range(1, 49))
ORACLE_SEEDS = list(range(101, 149))


def _schedule():
    kT = inputs.anneal_kT(N_ANNEAL, 3000.0, 300.0)
    return np.concatenate([kT, np.full(N_HOLD, inputs.K_B_EV * 300.0)])


def _model_coeffs():
    return inputs.pair_f32_coeffs(inputs.CONFIG2["coeff_seed"], NSH, S)


def _oracle_chain(seed):
    """One oracle chain: per-sweep energy and like-pair alpha over the window."""
    import oracle
    V = _model_coeffs()
    lat = oracle.Lattice(*DIMS, S)
    model = oracle.Model(oracle.PAIR_F32, NSH, V)
    occ = oracle.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, S), seed)
    kT = _schedule()
    E, A = [], []
    for t, kt in enumerate(kT):
        oracle.sweep(lat, model, occ, seed, t, 1, float(kt))
        if t >= len(kT) - WINDOW:
            E.append(oracle.total_energy(lat, model, occ))
            al = oracle.sro(lat, NSH, occ)
            A.append([al[m, p, p] for m in range(NSH) for p in range(S)])
    return float(np.mean(E)), np.mean(np.array(A), axis=0)


@pytest.fixture(scope="module")
def oracle_results():
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(ORACLE_SEEDS), max(1, mp.cpu_count()))) as pool:
        res = pool.map(_oracle_chain, ORACLE_SEEDS)
    return np.array([r[0] for r in res]), np.array([r[1] for r in res])


@pytest.fixture(scope="module")
def smc(oracle_results):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08250_gb300 import build, smc as s
    build.build()
    s.lib()
    return s


def test_anneal_window_means_agree_with_the_oracle(smc, oracle_results):
    V = _model_coeffs()
    lat = smc.Lattice(*DIMS, S)
    model = smc.Model(smc.PAIR_F32, NSH, V)
    kT = _schedule()
    dev = torch.device("cuda:0")
    gE, gA = [], []
    for seed in GPU_SEEDS:
        occ = torch.empty(lat.nsites, dtype=torch.int8, device=dev)
        smc.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, S), seed, occ)
        e = torch.zeros(WINDOW, dtype=torch.float64, device=dev)
        a = torch.zeros(WINDOW, NSH, S, S, dtype=torch.float64, device=dev)
        n0 = len(kT) - WINDOW
        smc.sweep(lat, model, occ, seed, 0, n0, kT[:n0])
        for i in range(WINDOW):
            smc.sweep(lat, model, occ, seed, n0 + i, 1, kT[n0 + i])
            smc.energy(lat, model, occ, e=e[i:i + 1])
            smc.sro(lat, NSH, occ, alpha=a[i])
        smc.check()
        gE.append(float(e.mean().item()))
        al = a.cpu().numpy()
        gA.append([al[:, m, p, p].mean() for m in range(NSH) for p in range(S)])
    gE, gA = np.array(gE), np.array(gA)
    oE, oA = oracle_results

    def check(g, o, what):
        se = math.sqrt(g.var(ddof=1) / len(g) + o.var(ddof=1) / len(o))
        z = (g.mean() - o.mean()) / se if se > 0 else 0.0
        assert abs(g.mean() - o.mean()) <= 3 * se + 1e-12, (what, g.mean(), o.mean(), se, z)

    check(gE, oE, "energy")
    for j in range(NSH * S):
        check(gA[:, j], oA[:, j], f"alpha shell {j // S + 1} species {j % S}")
