"""The fluctuation formula for parameter derivatives of canonical averages,
d<A>/dtheta = -beta (<A dE/dtheta> - <A><dE/dtheta>), pinned by exact
enumeration of the 16-site binary lattice (finite differences of the
enumerated average), and the binding's parameter-vector layout (CPU)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs

torch = pytest.importorskip("torch")


def enumerate_16_site(V, S=2):
    """All C(16, 8) equiatomic configurations of the 2x2x2-cell box: energy,
    SRO and dE/dtheta of each (oracle, FP64)."""
    lat = oracle.Lattice(2, 2, 2, S)
    model = oracle.Model(oracle.PAIR_F32, nshells=V.shape[0], v=V)
    E, A, G = [], [], []
    for ones in itertools.combinations(range(16), 8):
        occ = np.zeros(16, dtype=np.int8)
        occ[list(ones)] = 1
        E.append(oracle.total_energy(lat, model, occ))
        A.append(oracle.sro(lat, V.shape[0], occ))
        G.append(oracle.energy_grad(lat, model, occ))
    return np.array(E), np.array(A), np.array(G)


def boltzmann_mean(E, X, beta):
    w = np.exp(-beta * (E - E.min()))
    w /= w.sum()
    return np.tensordot(w, X, axes=(0, 0)), w


@pytest.mark.parametrize("kT", [0.025, 0.1])
def test_fluctuation_formula_equals_enumerated_derivative(kT):
    V = inputs.pair_f32_coeffs(3, 2, 2).astype(np.float64)
    E, A, G = enumerate_16_site(V.astype(np.float32))
    beta = 1.0 / kT
    meanA, w = boltzmann_mean(E, A, beta)
    meanG = w @ G
    cov = np.tensordot(w, A[..., None] * G[:, None, None, None, :], axes=(0, 0)) - meanA[..., None] * meanG
    formula = -beta * cov
    # E is linear in theta (E = theta . G), so theta + h e_j moves E by h G_j exactly
    h = 1e-5
    for j in range(G.shape[1]):
        ap, _ = boltzmann_mean(E + h * G[:, j], A, beta)
        am, _ = boltzmann_mean(E - h * G[:, j], A, beta)
        fd = (ap - am) / (2 * h)
        assert np.allclose(fd, formula[..., j], rtol=1e-5, atol=1e-7), j


def test_observable_gradient_is_the_sample_covariance():
    from paper_2604_08250_gb300 import smc
    rng = np.random.default_rng(1)
    A = rng.normal(size=(500, 2, 3))
    G = rng.normal(size=(500, 4)) + A[:, 0, :1]
    beta = 7.0
    got = smc.observable_gradient(torch.tensor(A), torch.tensor(G), beta).numpy()
    Af = A.reshape(500, -1)
    want = -beta * ((Af - Af.mean(0)).T @ (G - G.mean(0)) / 500).reshape(2, 3, 4)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


def test_parameter_vector_layout_round_trips():
    from paper_2604_08250_gb300 import smc
    S, nsh = 5, 2
    V = inputs.pair_f32_coeffs(5, nsh, S)
    mlp = inputs.mlp_weights(4)
    w = {k: oracle._widen(mlp[k]) for k in ("w1", "b1", "w2", "b2", "w3")}
    theta = [V[m, p, q] for m in range(nsh) for p in range(S) for q in range(p, S)]
    theta = np.concatenate([np.array(theta, dtype=np.float64), w["w1"], w["b1"], w["w2"], w["b2"], w["w3"], [0.5]])
    assert theta.size == smc.n_pair_params(nsh, S) + 5569
    model = smc.model_from_theta(smc.PAIR_F32_MLP_BF16, nsh, S, theta)
    assert np.array_equal(model.v, V)
    for k in ("w1", "w2", "w3"):  # BF16 values survive exactly
        assert np.array_equal(model.mlp[k], mlp[k].reshape(-1))
    assert model._c.mlp_b3 == 0.5
    # rounding to BF16 is to nearest
    t2 = theta.copy()
    k0 = smc.n_pair_params(nsh, S)
    t2[k0:k0 + 4] = [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -9]
    m2 = smc.model_from_theta(smc.PAIR_F32_MLP_BF16, nsh, S, t2)
    # BF16 spacing at 1 is 2^-7: ties go to the even pattern, the rest to the nearest
    assert list(m2.mlp["w1"][:4]) == [0x3F80, 0x3F82, 0x3F81, 0x3F80]
    with pytest.raises(ValueError):
        smc.model_from_theta(smc.MLP_BF16, 0, S, theta)
    assert math.isfinite(float(theta.sum()))
