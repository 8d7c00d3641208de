"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds workload definitions only (random coefficient draws,
compositions, MLP weights, temperature schedules, replica sizes).  It contains
none of the Monte Carlo arithmetic, and imports neither the CUDA binding nor
the oracle.  The paper's workloads (an FCC high-entropy alloy with trained
qSRO / MLPNet models, Sec. IV) need trained weights that are not available;
these draws stand in for them with the same shapes and magnitudes.
"""
from __future__ import annotations

import numpy as np

K_B_EV = 8.617333262e-5  # Boltzmann constant, eV/K (CODATA 2018)


def equiatomic_counts(nsites: int, nspecies: int) -> np.ndarray:
    """floor(N/S) sites per species, the remainder given to species 0..r-1."""
    base, rem = divmod(int(nsites), int(nspecies))
    c = np.full(nspecies, base, dtype=np.int64)
    c[:rem] += 1
    return c


def dirichlet_counts(nsites: int, nspecies: int, seed: int, alpha: float = 5.0) -> np.ndarray:
    """Composition p ~ Dir(alpha 1_S) from default_rng(seed), turned into
    integer counts by the largest-remainder rule."""
    rng = np.random.default_rng(seed)
    p = rng.dirichlet(np.full(nspecies, alpha))
    raw = p * nsites
    c = np.floor(raw).astype(np.int64)
    short = int(nsites - c.sum())
    order = np.argsort(-(raw - c), kind="stable")
    c[order[:short]] += 1
    return c


# The paper's alloy Fe29 Co29 Ni28 Al7 Ti7 (Sec. IV-C), species 0-4 in that order.
HEA_FRACTIONS = (0.29, 0.29, 0.28, 0.07, 0.07)


def fraction_counts(nsites: int, fractions) -> np.ndarray:
    """Integer counts of the given composition by the largest-remainder rule."""
    raw = np.asarray(fractions, dtype=np.float64) / float(np.sum(fractions)) * nsites
    c = np.floor(raw).astype(np.int64)
    short = int(nsites - c.sum())
    order = np.argsort(-(raw - c), kind="stable")
    c[order[:short]] += 1
    return c


def _symmetric(unique: np.ndarray, nshells: int, S: int, dtype) -> np.ndarray:
    v = np.zeros((nshells, S, S), dtype=dtype)
    t = 0
    for m in range(nshells):
        for p in range(S):
            for q in range(p, S):
                v[m, p, q] = v[m, q, p] = unique[t]
                t += 1
    return v


def pair_int_coeffs(seed: int, nshells: int = 2, nspecies: int = 2, lo: int = -500, hi: int = 500) -> np.ndarray:
    """Integer pair coefficients V_m(p,q) (units of 0.1 meV), uniform in
    [lo, hi], one draw per unordered pair, shell-major then p <= q."""
    rng = np.random.default_rng(seed)
    n = nshells * nspecies * (nspecies + 1) // 2
    return _symmetric(rng.integers(lo, hi + 1, size=n), nshells, nspecies, np.int32)


def pair_f32_coeffs(seed: int, nshells: int = 2, nspecies: int = 5, sigma_ev: float = 0.020) -> np.ndarray:
    """FP32 pair coefficients V_m(p,q) ~ N(0, sigma) eV, symmetric."""
    rng = np.random.default_rng(seed)
    n = nshells * nspecies * (nspecies + 1) // 2
    return _symmetric(rng.normal(0.0, sigma_ev, size=n), nshells, nspecies, np.float64).astype(np.float32)


def qsro_coeffs(seed: int, nshells: int = 2, nspecies: int = 5, sigma_v_ev: float = 0.100,
                sigma_w_ev: float = 0.050, c_ev: float = -4.0):
    """qSRO parameters (V_m^{pp'} symmetric [nshells][S][S], W_m^p
    [nshells][S], C), FP32: V ~ N(0, sigma_v), W ~ N(0, sigma_w) eV.  Site
    energies weigh pair fractions (sums of 1), so these are the pair model's
    coefficients times a coordination number in size."""
    rng = np.random.default_rng(seed)
    n = nshells * nspecies * (nspecies + 1) // 2
    V = _symmetric(rng.normal(0.0, sigma_v_ev, size=n), nshells, nspecies, np.float64).astype(np.float32)
    W = rng.normal(0.0, sigma_w_ev, size=(nshells, nspecies)).astype(np.float32)
    return V, W, float(np.float32(c_ev))


def ordering_coeffs_b2() -> np.ndarray:
    """Binary ordering interactions whose ground state is B2 (CsCl):
    unlike first neighbours attract, like second neighbours attract."""
    v = np.zeros((2, 2, 2), dtype=np.int32)
    v[0] = [[100, -100], [-100, 100]]
    v[1] = [[-50, 50], [50, -50]]
    return v


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit patterns, round to nearest even."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def mlp_weights(seed: int, n_in: int = 20, n_hid: int = 64, out_scale: float = 0.01) -> dict:
    """Xavier-uniform weights U(+-sqrt(6/(fan_in+fan_out))) from
    default_rng(seed), rounded to BF16; zero biases.  The output layer is
    multiplied by out_scale before rounding so that site energies are a few
    meV (untrained Xavier weights give O(0.5 eV) per site)."""
    rng = np.random.default_rng(seed)

    def xavier(fan_out, fan_in):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-lim, lim, size=(fan_out, fan_in))

    w1 = xavier(n_hid, n_in)
    w2 = xavier(n_hid, n_hid)
    w3 = xavier(1, n_hid)[0] * out_scale
    return {
        "w1": to_bf16_bits(w1.astype(np.float32)).reshape(-1),
        "w2": to_bf16_bits(w2.astype(np.float32)).reshape(-1),
        "w3": to_bf16_bits(w3.astype(np.float32)).reshape(-1),
        "b1": np.zeros(n_hid, dtype=np.float32),
        "b2": np.zeros(n_hid, dtype=np.float32),
        "b3": 0.0,
    }


def mlpnet_weights(seed: int, n_in: int = 20, n_hid: int = 96, out_scale: float = 0.01,
                   bias_sigma: float = 0.05) -> dict:
    """MLPNet at the paper's shape (20 -> 96 -> 96 -> 96 -> 1, ReLU): He-uniform
    weights U(+-sqrt(6/fan_in)) from default_rng(seed) rounded to BF16, FP32
    biases N(0, bias_sigma) (so the bias path is exercised), output layer
    multiplied by out_scale before rounding (site energies of a few meV)."""
    rng = np.random.default_rng(seed)

    def he(fan_out, fan_in):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=(fan_out, fan_in))

    w0 = he(n_hid, n_in)
    w1 = he(n_hid, n_hid)
    w2 = he(n_hid, n_hid)
    w3 = he(1, n_hid)[0] * out_scale
    bias = [rng.normal(0.0, bias_sigma, n_hid).astype(np.float32) for _ in range(3)]
    return {
        "w0": to_bf16_bits(w0.astype(np.float32)).reshape(-1),
        "w1": to_bf16_bits(w1.astype(np.float32)).reshape(-1),
        "w2": to_bf16_bits(w2.astype(np.float32)).reshape(-1),
        "w3": to_bf16_bits(w3.astype(np.float32)).reshape(-1),
        "b0": bias[0],
        "b1": bias[1],
        "b2": bias[2],
        "b3": float(np.float32(rng.normal(0.0, 0.001))),
    }


def anneal_kT(nsweeps: int = 1000, t_start: float = 3000.0, t_end: float = 300.0) -> np.ndarray:
    """Linear anneal T_t = t_start + (t_end - t_start) t/(nsweeps-1), kT in eV."""
    t = np.arange(nsweeps, dtype=np.float64)
    T = t_start + (t_end - t_start) * t / max(nsweeps - 1, 1)
    return K_B_EV * T


def ladder_kT(nrep: int = 64, t_min: float = 300.0, t_max: float = 3000.0) -> np.ndarray:
    """Geometric temperature ladder T_r = t_min (t_max/t_min)^(r/(R-1)), kT in eV."""
    r = np.arange(nrep, dtype=np.float64)
    return K_B_EV * t_min * (t_max / t_min) ** (r / max(nrep - 1, 1))


def batched_edges(seed: int, nrep: int = 64, lo: int = 8, hi: int = 24) -> np.ndarray:
    """Uneven cubic replica edges (cells): 4 * integers(lo, hi] from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return 4 * rng.integers(lo, hi + 1, size=nrep)


# Workloads (BCC; N = 2 * cells).  kT values in eV.
CONFIG1 = dict(name="bcc8_binary_int_pair", cells=(8, 8, 8), nspecies=2, nshells=2,
               coeff_seed=1, mc_seed=1, kT_ev=0.025, unit_ev=1e-4, nsweeps=100)
CONFIG2 = dict(name="bcc128_quinary_f32_pair_anneal", cells=(128, 128, 128), nspecies=5, nshells=2,
               coeff_seed=2, mc_seed=1, nsweeps=1000, t_start=3000.0, t_end=300.0)
CONFIG3 = dict(name="batched64_quinary_f32_pair_ladder", nrep=64, nspecies=5, nshells=2,
               edge_seed=3, coeff_seed=3, mc_seed=1, nsweeps=500, t_min=300.0, t_max=3000.0)
CONFIG4 = dict(name="bcc256_quinary_mlp_bf16", cells=(256, 256, 256), nspecies=5,
               comp_seed=4, mlp_seed=4, mc_seed=1, nsweeps=200, T=800.0)
CONFIG5 = dict(name="bcc512_quinary_pair_mlp_grad", cells=(512, 512, 512), nspecies=5, nshells=2,
               coeff_seed=5, mlp_seed=4, mc_seed=1, nsamples=200, T=600.0, fd_cells=(16, 16, 16))
