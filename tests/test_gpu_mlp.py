"""GPU parity of the MLP paths (BF16 tensor-core site energies) against the
FP64 oracle, through the C ABI.

The BF16 path cannot match FP64 bit for bit.  Every trial's dE is checked
twice: tightly against an FP64 emulation of the BF16 evaluation order
(tests/helpers.mlp_bf16_emulation: layer-1 activations rounded to BF16), with
a bound from FP32 accumulation, the tanh approximation and rounding-boundary
cases; and against the FP64 oracle within the worst-case bound of the BF16
arithmetic (tests/helpers.mlp_error_bound), with the sign of dE agreeing
wherever |dE| exceeds it.  A decision may differ from the oracle's only where
the acceptance threshold lies between the two values.  The sweep kernel
(cached pre-swap energies) must reproduce the trace kernel (recomputed
energies) bit for bit.  Error statistics go to
$SMC_STATS_DIR/mlp_dE_errors.json when that is set."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs
from tests import helpers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K_B = inputs.K_B_EV
_STATS = {}


@pytest.fixture(scope="module")
def smc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08250_gb300 import build, smc as s
    build.build()
    s.lib()
    yield s
    d = os.environ.get("SMC_STATS_DIR")
    if d and _STATS:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "mlp_dE_errors.json"), "w") as f:
            json.dump(_STATS, f, indent=1, sort_keys=True)


def dev():
    return torch.device("cuda:0")


def make_models(smc, kind, S=5, mlp_seed=4, coeff_seed=5, nshells=2, out_scale=0.01, biases=False):
    mlp = inputs.mlp_weights(mlp_seed, out_scale=out_scale)
    if biases:  # exercise b1, b2, b3 as well (zero in the standard draw)
        rng = np.random.default_rng(mlp_seed + 100)
        mlp["b1"] = rng.normal(0, 0.3, 64).astype(np.float32)
        mlp["b2"] = rng.normal(0, 0.3, 64).astype(np.float32)
        mlp["b3"] = 0.0123
    V = inputs.pair_f32_coeffs(coeff_seed, nshells, S) if kind == smc.PAIR_F32_MLP_BF16 else None
    gm = smc.Model(kind, nshells=nshells if V is not None else 0, v=V, mlp=mlp)
    om = oracle.Model(oracle.PAIR_F32_MLP if V is not None else oracle.MLP, nshells=nshells if V is not None else 0,
                      v=V, mlp=mlp)
    w = {k: oracle._widen(mlp[k]).reshape(64, -1) if k in ("w1", "w2") else oracle._widen(mlp[k])
         for k in ("w1", "w2", "w3", "b1", "b2")}
    w["b3"] = float(mlp["b3"])
    return gm, om, w, V


def start_state(smc, dims, S, seed, counts_seed=4):
    """The oracle's start state on the device, and on the host (the oracle
    never reads a configuration the GPU produced)."""
    N = 2 * dims[0] * dims[1] * dims[2]
    counts = inputs.dirichlet_counts(N, S, counts_seed)
    lat = smc.Lattice(*dims, S)
    ref = oracle.init_lattice(oracle.Lattice(*dims, S), counts, seed)
    return lat, torch.from_numpy(ref.copy()).to(dev()), counts, ref


def trial_reference(occ_h, dims, a, b, w, dE64, V=None):
    """Per trial (a[t], b[t]) on occ_h: the BF16-emulated dE (the FP64 pair
    part included), the bound on |dE_GPU - dE_emulated| and the worst-case
    bound on |dE_GPU - dE_FP64|."""
    nt = len(a)
    oms = [helpers.omega(int(a[t]), int(b[t]), dims) for t in range(nt)]
    Xpre = helpers.mlp_features(occ_h, dims, np.concatenate(oms))
    Xpost = np.concatenate([helpers.mlp_features(occ_h, dims, oms[t], swap=(int(a[t]), int(b[t])))
                            for t in range(nt)])
    e_pre, f_pre = helpers.mlp_error_bound(Xpre, w)
    e_post, f_post = helpers.mlp_error_bound(Xpost, w)
    g_pre, gb_pre = helpers.mlp_bf16_emulation(Xpre, w)
    g_post, gb_post = helpers.mlp_bf16_emulation(Xpost, w)

    def per(v):
        return v.reshape(nt, -1).sum(axis=1)

    sum_err = 80 * 2.0 ** -24 * per(np.abs(f_pre) + np.abs(f_post))
    pair_err = 0.0
    if V is not None:  # <= 26 FP32 products of |count| <= 8 and |D| <= 2 max|V|
        pair_err = 64 * 2.0 ** -24 * 26 * 8 * 2 * float(np.abs(V).max())
    loose = (per(e_pre + e_post) + sum_err + pair_err) * 1.05 + 1e-12
    tight = (per(gb_pre + gb_post) + sum_err + pair_err) * 1.05 + 1e-12
    emu = np.asarray(dE64) - per(f_post - f_pre) + per(g_post - g_pre)
    return emu, tight, loose


def threshold(seed, sweep, a, kT, replica=0):
    """-kT ln u of the trial at site a, u = (r + 1/2) 2^-29 from its Philox word."""
    w = oracle.philox4x32_10([a >> 2, replica, sweep & 0xFFFFFFFF, sweep >> 32],
                             [seed & 0xFFFFFFFF, seed >> 32])[a & 3]
    r = int(w) & ((1 << 29) - 1)
    return -kT * math.log((r + 0.5) * 2.0 ** -29)


def record(name, err64, err_emu, loose, flips, n):
    err64, err_emu = np.asarray(err64), np.asarray(err_emu)
    _STATS[name] = {"trials": int(n), "max_abs_err_vs_fp64_eV": float(np.abs(err64).max()),
                    "rms_err_vs_fp64_eV": float(np.sqrt(np.mean(err64 ** 2))),
                    "max_abs_err_vs_bf16_emulation_eV": float(np.abs(err_emu).max()),
                    "rms_err_vs_bf16_emulation_eV": float(np.sqrt(np.mean(err_emu ** 2))),
                    "median_worst_case_bound_eV": float(np.median(loose)), "decision_flips": int(flips)}


@pytest.mark.parametrize("dims,kind,T,biases", [((16, 16, 16), 2, 800.0, False), ((24, 16, 8), 2, 300.0, True),
                                                ((8, 8, 8), 2, 800.0, False), ((16, 8, 12), 3, 600.0, False)])
def test_mlp_lockstep_against_oracle(smc, dims, kind, T, biases):
    """Every trial of a full sweep: |dE_GPU - dE_emulated| within the tight
    bound, |dE_GPU - dE_FP64| within the worst-case bound, the sign agreeing
    beyond it; a decision flip only where the acceptance threshold lies between
    the oracle's dE and the GPU's (the run continues from the oracle's state)."""
    S, seed, kT = 5, 11, K_B * T
    gm, om, w, V = make_models(smc, kind, biases=biases)
    lat, occ, _, ref = start_state(smc, dims, S, seed)
    olat = oracle.Lattice(*dims, S)
    nt = lat.nsites // 128
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    acc = torch.zeros(nt, dtype=torch.uint8, device=dev())
    errs, emus, bnds, flips, n = [], [], [], 0, 0
    for k in range(128):
        occ_h = ref.copy()  # the pre-step state, the oracle's
        smc.ministep_trace(lat, gm, occ, seed, 0, k, kT, dE, acc)
        smc.check()
        d_o, a_o, a, b = oracle.ministep_trace(olat, om, ref, seed, 0, k, kT)
        d_g = dE.cpu().numpy().astype(np.float64)
        a_g = acc.cpu().numpy().astype(bool)
        emu, tight, loose = trial_reference(occ_h, dims, a, b, w, d_o, V)
        e_emu = d_g - emu
        err = d_g - d_o
        assert np.all(np.abs(err) <= loose)
        big = np.abs(d_o) > loose
        assert np.all(np.sign(d_g[big]) == np.sign(d_o[big]))
        for t in np.flatnonzero(a_g != a_o):
            thr = threshold(seed, 0, int(a[t]), kT)
            slack = abs(err[t]) * (1 + 1e-6)
            assert abs(d_o[t] - thr) <= slack + 1e-6 * thr or abs(d_o[t]) <= slack, (k, t, d_o[t], thr)
            flips += 1
        if np.any(a_g != a_o):  # the GPU continues from the oracle's state
            occ.copy_(torch.from_numpy(ref.copy()).to(dev()))
        errs.append(err)
        emus.append(e_emu)
        bnds.append(loose)
        n += nt
    errs, emus = np.concatenate(errs), np.concatenate(emus)
    record(f"lockstep_{dims[0]}x{dims[1]}x{dims[2]}_kind{kind}_T{int(T)}", errs, emus, np.concatenate(bnds),
           flips, n)
    # the GPU follows the BF16 evaluation order: its departures from the
    # emulation (tanh approximation, FP32 accumulation) are well below the
    # BF16 quantisation itself, which a wrong feature or zone would exceed
    quant = np.sqrt(np.mean((errs - emus) ** 2))
    assert np.sqrt(np.mean(emus ** 2)) <= 0.5 * quant


@pytest.mark.parametrize("dims,kind", [((16, 16, 16), 2), ((24, 16, 8), 2), ((8, 8, 8), 2), ((16, 8, 12), 3),
                                       ((8, 12, 20), 3), ((1024, 8, 8), 2), ((300, 12, 8), 3)])
def test_mlp_sweep_kernel_equals_trace_kernel(smc, dims, kind):
    """Two sweeps of the persistent kernel (cached energies, staged windows,
    neighbour flags) == 256 lock-step mini-steps (recomputed energies): same
    occupancy, same accept count, e_acc equal to the sum of the traced dE up
    to FP64 summation order."""
    S, seed, kT = 5, 21, K_B * 800.0
    gm, _, _, _ = make_models(smc, kind)
    lat, occ, counts, _ = start_state(smc, dims, S, seed)
    occ2 = occ.clone()
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.sweep(lat, gm, occ, seed, 5, 2, kT, e_acc=e_acc, n_acc=n_acc)
    smc.check()
    nt = lat.nsites // 128
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    acc = torch.zeros(nt, dtype=torch.uint8, device=dev())
    tot, cnt, mag = 0.0, 0, 0.0
    for t in range(2):
        for k in range(128):
            smc.ministep_trace(lat, gm, occ2, seed, 5 + t, k, kT, dE, acc)
            d = dE.cpu().numpy().astype(np.float64)
            a = acc.cpu().numpy().astype(bool)
            tot += d[a].sum()
            mag += np.abs(d[a]).sum()
            cnt += int(a.sum())
    smc.check()
    assert torch.equal(occ, occ2)
    assert int(n_acc.item()) == cnt
    assert abs(e_acc.item() - tot) <= 1e-12 * mag + 1e-15
    assert np.array_equal(np.bincount(occ.cpu().numpy(), minlength=S), counts)


@pytest.mark.parametrize("dims,kind,biases", [((8, 8, 8), 2, False), ((16, 8, 12), 2, True), ((12, 8, 8), 3, False)])
def test_mlp_energy_matches_oracle(smc, dims, kind, biases):
    """smc_energy = sum_i f(x_i) (+ pair energy) within the summed per-site bound."""
    S, seed = 5, 3
    gm, om, w, V = make_models(smc, kind, biases=biases)
    lat, occ, _, occ_h = start_state(smc, dims, S, seed)
    e = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.energy(lat, gm, occ, e)
    smc.check()
    want = oracle.total_energy(oracle.Lattice(*dims, S), om, occ_h)
    eb, f = helpers.mlp_error_bound(helpers.mlp_features(occ_h, dims, np.arange(lat.nsites)), w)
    tol = eb.sum() + lat.nsites * 2.0 ** -40 * np.abs(f).sum() + 1e-12
    if V is not None:
        tol += 1e-9 * lat.nsites * float(np.abs(V).max()) * 26
    assert abs(e.item() - want) <= tol, (e.item(), want, tol)


def test_mlp_energy_bookkeeping_and_composition(smc):
    """After sweeps, E(after) - E(before) equals the accumulated dE within the
    bounds of both, and the composition is unchanged."""
    dims, S, seed, kT = (16, 16, 16), 5, 8, K_B * 800.0
    gm, _, w, _ = make_models(smc, 2)
    lat, occ, counts, _ = start_state(smc, dims, S, seed)
    e0 = torch.zeros(1, dtype=torch.float64, device=dev())
    e1 = torch.zeros(1, dtype=torch.float64, device=dev())
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    occ0 = occ.cpu().numpy()
    smc.energy(lat, gm, occ, e0)
    smc.sweep(lat, gm, occ, seed, 0, 4, kT, e_acc=e_acc, n_acc=n_acc)
    smc.energy(lat, gm, occ, e1)
    smc.check()
    occ1 = occ.cpu().numpy()
    assert np.array_equal(np.bincount(occ1, minlength=S), counts)
    assert 0 < n_acc.item() < 4 * lat.nsites
    b0, _ = helpers.mlp_error_bound(helpers.mlp_features(occ0, dims, np.arange(lat.nsites)), w)
    b1, _ = helpers.mlp_error_bound(helpers.mlp_features(occ1, dims, np.arange(lat.nsites)), w)
    # each accepted trial's dE error is at most ~80 site bounds of typical size
    per_trial = 80 * 2 * float(max(b0.max(), b1.max()))
    tol = b0.sum() + b1.sum() + n_acc.item() * per_trial
    assert abs((e1.item() - e0.item()) - e_acc.item()) <= tol


def test_mlp_rejects_unsupported_shapes(smc):
    gm, _, _, _ = make_models(smc, 2)
    lat = smc.Lattice(6, 8, 8, 5)
    occ = torch.zeros(lat.nsites, dtype=torch.int8, device=dev())
    with pytest.raises(smc.SMCError) as ei:
        smc.sweep(lat, gm, occ, 1, 0, 1, 0.05)
    assert ei.value.code == smc.SMC_ERR_UNSUPPORTED
    lat6 = smc.Lattice(8, 8, 8, 6)
    with pytest.raises(smc.SMCError) as ei:
        smc.sweep(lat6, gm, torch.zeros(lat6.nsites, dtype=torch.int8, device=dev()), 1, 0, 1, 0.05)
    assert ei.value.code == smc.SMC_ERR_ARG


def test_config4_full_size_sampled(smc):
    """The MLP workload at full size (256^3 cells, 33.5 M sites, Dirichlet
    quinary, 800 K): one sweep of the persistent kernel equals 128 lock-step
    mini-steps bit for bit; 256 sampled trials of one mini-step are within
    their bound of the FP64 oracle's dE; the composition is unchanged."""
    c = inputs.CONFIG4
    dims, S = c["cells"], c["nspecies"]
    kT = K_B * c["T"]
    seed = c["mc_seed"]
    gm, om, w, _ = make_models(smc, 2, mlp_seed=c["mlp_seed"])
    lat, occ, counts, ref = start_state(smc, dims, S, seed, counts_seed=c["comp_seed"])
    occ2 = occ.clone()
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.sweep(lat, gm, occ, seed, 0, 1, kT, n_acc=n_acc)
    smc.check()
    nt = lat.nsites // 128
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    acc = torch.zeros(nt, dtype=torch.uint8, device=dev())
    k_s = 77
    olat = oracle.Lattice(*dims, S)
    nv = oracle.shell_vectors(1)
    rng = np.random.default_rng(0)
    for k in range(128):
        smc.ministep_trace(lat, gm, occ2, seed, 0, k, kT, dE, acc)
    smc.check()
    assert torch.equal(occ, occ2)
    assert np.array_equal(np.bincount(occ.cpu().numpy(), minlength=S), counts)
    assert 0 < n_acc.item() < lat.nsites
    # mini-step k_s on the oracle's start state (a valid input to any mini-step)
    occ_h = ref
    occ2.copy_(torch.from_numpy(ref.copy()).to(dev()))
    smc.ministep_trace(lat, gm, occ2, seed, 0, k_s, kT, dE, acc)
    smc.check()
    d_g = dE.cpu().numpy().astype(np.float64)
    # sampled trials of mini-step k_s against the oracle
    nx, ny, nz = dims
    NLx, NLy = nx // 4, ny // 4
    dx, dy, dz, sub = k_s % 4, (k_s // 4) % 4, (k_s // 16) % 4, k_s // 64
    cs = rng.choice(nt, 256, replace=False)
    a_l, b_l, d_o = [], [], []
    for cidx in cs:
        cx, cy, cz = cidx % NLx, (cidx // NLx) % NLy, cidx // (NLx * NLy)
        a = ((sub * nz + 4 * cz + dz) * ny + 4 * cy + dy) * nx + 4 * cx + dx
        wd = oracle.philox4x32_10([a >> 2, 0, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])[a & 3]
        b = oracle.neighbor(olat, a, nv[int(wd) >> 29])
        a_l.append(a)
        b_l.append(b)
        d_o.append(oracle.delta_e(olat, om, occ_h, a, b))
    d_o = np.array(d_o)
    emu, tight, loose = trial_reference(occ_h, dims, a_l, b_l, w, d_o)
    assert np.all(np.abs(d_g[cs] - d_o) <= loose)
    assert np.sqrt(np.mean((d_g[cs] - emu) ** 2)) <= 0.5 * np.sqrt(np.mean((emu - d_o) ** 2))
    record("config4_256cubed_sampled", d_g[cs] - d_o, d_g[cs] - emu, loose, 0, len(cs))


GRAD_REL = 2.0 ** -7 + 2.0 ** -9  # two BF16 roundings per term, sigmoid approximations, FP32 sums


@pytest.mark.parametrize("dims,kind,ctas", [((8, 8, 8), 2, 0), ((12, 8, 8), 3, 0), ((2, 2, 2), 2, 0),
                                            ((56, 56, 56), 2, 1)])
def test_mlp_gradient_matches_oracle(smc, dims, kind, ctas):
    """dE/dtheta (pair part exact, then the 5569 MLP parameters) against the
    oracle's FP64 back-propagation: every MLP entry within GRAD_REL of the sum
    of the magnitudes of its terms; dE/db3 = N exactly.  The 56^3 case with
    one CTA per SM runs enough blocks per CTA to exercise the FP64 flushes."""
    S = 5
    gm, om, w, V = make_models(smc, kind, biases=True)
    lat, occ, _, occ_h = start_state(smc, dims, S, 17)
    n = smc.grad_size(lat, gm)
    g = torch.zeros(n, dtype=torch.float32, device=dev())
    try:
        smc.set_tuning(ctas_per_sm=ctas)
        smc.energy_grad(lat, gm, occ, g)
        smc.check()
    finally:
        smc.set_tuning()
    want = oracle.energy_grad(oracle.Lattice(*dims, S), om, occ_h)
    got = g.cpu().numpy().astype(np.float64)
    npair = n - 5569
    assert np.array_equal(got[:npair], want[:npair])
    scale = helpers.mlp_grad_abs_terms(helpers.mlp_features(occ_h, dims, np.arange(lat.nsites)), w)
    err = np.abs(got[npair:] - want[npair:])
    assert np.all(err <= GRAD_REL * scale + 1e-7), (np.flatnonzero(err > GRAD_REL * scale + 1e-7)[:5],
                                                     (err / (scale + 1e-30)).max())
    assert got[-1] == lat.nsites
    rel = float(np.linalg.norm(got[npair:] - want[npair:]) / np.linalg.norm(want[npair:]))
    _STATS[f"grad_{dims[0]}x{dims[1]}x{dims[2]}_kind{kind}"] = {
        "norm_rel_err": rel, "max_err_over_term_scale": float((err / (scale + 1e-30)).max())}
    assert rel < 1e-3
