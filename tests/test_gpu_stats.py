"""GPU chains against exact enumeration, and the differentiable energy.

On the 16-site binary lattice (2x2x2 cells) the canonical averages <E>,
<alpha> and d<alpha>/dtheta are known exactly by enumeration; GPU sweeps must
reproduce them within 3 batch-means standard errors, the derivative through
the fluctuation formula on per-sample dE/dtheta from smc_energy_grad.
SMCEnergy must give smc_energy forward and smc_energy_grad backward."""
import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs
from tests.test_observable_gradient import boltzmann_mean, enumerate_16_site

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08250_gb300 import build, smc as s
    build.build()
    s.lib()
    return s


def batch_se(x, nb=20):
    """Mean over samples and its batch-means standard error (axis 0)."""
    x = np.asarray(x)
    b = x[: len(x) // nb * nb].reshape(nb, -1, *x.shape[1:]).mean(axis=1)
    return x.mean(axis=0), b.std(axis=0, ddof=1) / np.sqrt(nb)


@pytest.mark.parametrize("kT", [0.06, 0.15])
def test_gpu_chain_matches_enumeration_16_site(smc, kT):
    """sigma = 5 meV coefficients: at these temperatures the chain visits many
    energy levels, so fluctuations are not a few rare excursions."""
    S, nsh, seed = 2, 2, 5
    V = inputs.pair_f32_coeffs(3, nsh, S, sigma_ev=0.005)
    E, A, G = enumerate_16_site(V)
    beta = 1.0 / kT
    mA, w = boltzmann_mean(E, A, beta)
    mE = w @ E
    mG = w @ G
    dA = -beta * (np.tensordot(w, A[..., None] * G[:, None, None, None, :], axes=(0, 0)) - mA[..., None] * mG)

    lat = smc.Lattice(2, 2, 2, S)
    gm = smc.Model(smc.PAIR_F32, nshells=nsh, v=V)
    occ = torch.empty(16, dtype=torch.int8, device="cuda")
    smc.init_lattice(lat, [8, 8], seed, occ)
    burn, n = 1000, 40000
    smc.sweep(lat, gm, occ, seed, 0, burn, kT)
    P = smc.grad_size(lat, gm)
    Es = torch.zeros(n, dtype=torch.float64, device="cuda")
    As = torch.zeros(n, nsh, S, S, dtype=torch.float64, device="cuda")
    Gs = torch.zeros(n, P, dtype=torch.float32, device="cuda")
    for i in range(n):
        smc.sweep(lat, gm, occ, seed, burn + i, 1, kT)
        smc.energy(lat, gm, occ, Es[i:i + 1])
        smc.sro(lat, nsh, occ, alpha=As[i])
        smc.energy_grad(lat, gm, occ, Gs[i])
    smc.check()
    Es, As, Gs = Es.cpu().numpy(), As.cpu().numpy(), Gs.cpu().numpy().astype(np.float64)
    m, se = batch_se(Es)
    assert abs(m - mE) <= 3 * se + 1e-9, (m, mE, se, (m - mE) / se)
    a01 = As[:, 0, 0, 1]
    m, se = batch_se(a01)
    assert abs(m - mA[0, 0, 1]) <= 3 * se + 1e-9, (m, mA[0, 0, 1], se, (m - mA[0, 0, 1]) / se)
    # d<alpha_1^{01}>/dtheta from the samples; standard error from contiguous batches
    nb = 20
    per = np.stack([smc.observable_gradient(torch.tensor(a[:, None]), torch.tensor(g), beta).numpy()[0]
                    for a, g in zip(a01.reshape(nb, -1), Gs.reshape(nb, -1, Gs.shape[1]))])
    est = smc.observable_gradient(torch.tensor(a01[:, None]), torch.tensor(Gs), beta).numpy()[0]
    se = per.std(axis=0, ddof=1) / np.sqrt(nb)
    want = dA[0, 0, 1]
    assert np.all(np.abs(est - want) <= 3 * se + 1e-6 * np.abs(want).max() + 1e-9), (est, want, se, (est - want) / se)


@pytest.mark.parametrize("kind", [2, 3])
def test_smc_energy_autograd(smc, kind):
    dims, S, nsh = (8, 8, 8), 5, 2
    mlp = inputs.mlp_weights(4)
    V = inputs.pair_f32_coeffs(5, nsh, S)
    parts = []
    if kind == smc.PAIR_F32_MLP_BF16:
        parts.append(np.array([V[m, p, q] for m in range(nsh) for p in range(S) for q in range(p, S)]))
    parts += [oracle._widen(mlp[k]) for k in ("w1", "b1", "w2", "b2", "w3")] + [np.array([0.0])]
    theta = torch.tensor(np.concatenate(parts), dtype=torch.float64, requires_grad=True)
    n_sh = nsh if kind == smc.PAIR_F32_MLP_BF16 else 0
    lat = smc.Lattice(*dims, S)
    occ = torch.empty(lat.nsites, dtype=torch.int8, device="cuda")
    smc.init_lattice(lat, inputs.dirichlet_counts(lat.nsites, S, 4), 3, occ)
    E = smc.smc_energy_fn(theta, lat, occ, kind, n_sh)
    (g,) = torch.autograd.grad(E * 2.0, theta)
    model = smc.model_from_theta(kind, n_sh, S, theta.detach().numpy())
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    smc.energy(lat, model, occ, e)
    gg = torch.zeros(smc.grad_size(lat, model), dtype=torch.float32, device="cuda")
    smc.energy_grad(lat, model, occ, gg)
    assert float(E.detach()) == float(e.item())
    assert torch.equal(g, 2.0 * gg.double().cpu())
    if kind == smc.PAIR_F32_MLP_BF16:  # E is linear in the pair coefficients: central differences are exact
        npair = smc.n_pair_params(nsh, S)
        for j in (0, 7, npair - 1):
            h = 1e-3
            tp, tm = theta.detach().clone(), theta.detach().clone()
            tp[j] += h
            tm[j] -= h
            fd = (float(smc.smc_energy_fn(tp, lat, occ, kind, n_sh)) -
                  float(smc.smc_energy_fn(tm, lat, occ, kind, n_sh))) / (2 * h)
            assert abs(fd - float(gg[j])) <= 1e-3 * abs(float(gg[j])) + 1e-2
