"""Pins of the oracle's MLPNet (Sec. IV-B: 20 -> 96 -> 96 -> 96 -> 1, ReLU
after the input layer and each hidden layer, linear output) on CPU.

* Non-negative weights, biases and inputs keep every ReLU in its identity
  branch: f is then the composed affine map, computed here with matrix
  products.
* A layer whose weights are non-positive and biases negative outputs 0 on
  non-negative inputs: f reduces to the closed form of the layers after it
  (one case per layer, so a misplaced or missing ReLU fails).
* Without biases the network is positively homogeneous: f(c x) = c f(x).
* The site energy is f of the site's features (one-hot species and per-shell
  species counts), checked on a pure element where the features are known.
* Every incremental dE equals the change of the total energy (3-shell zone).
"""
import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs

H, NIN = 96, 20


def _net(w0, w1, w2, w3, b0, b1, b2, b3):
    return {"w0": w0.reshape(-1), "w1": w1.reshape(-1), "w2": w2.reshape(-1), "w3": w3.reshape(-1),
            "b0": b0, "b1": b1, "b2": b2, "b3": b3}


def _rand(rng, pos=True):
    f = (lambda a: np.abs(a)) if pos else (lambda a: a)
    w0 = f(rng.normal(0, 0.2, (H, NIN)))
    w1 = f(rng.normal(0, 0.1, (H, H)))
    w2 = f(rng.normal(0, 0.1, (H, H)))
    w3 = f(rng.normal(0, 0.1, H))
    b0, b1, b2 = (f(rng.normal(0, 0.1, H)) for _ in range(3))
    return w0, w1, w2, w3, b0, b1, b2


def test_affine_regime_is_the_composed_map():
    rng = np.random.default_rng(1)
    w0, w1, w2, w3, b0, b1, b2 = _rand(rng)
    m = oracle.Model(oracle.MLPNET, net=_net(w0, w1, w2, w3, b0, b1, b2, 0.25))
    for _ in range(20):
        x = np.abs(rng.normal(0, 3, NIN))
        want = w3 @ (w2 @ (w1 @ (w0 @ x + b0) + b1) + b2) + 0.25
        assert oracle.mlpnet_eval(m, x) == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("dead", [0, 1, 2])
def test_dead_layer_closed_forms(dead):
    rng = np.random.default_rng(10 + dead)
    w = list(_rand(rng))  # w0, w1, w2, w3, b0, b1, b2, all >= 0
    wi, bi = dead, 4 + dead
    w[wi] = -w[wi]
    w[bi] = -w[bi] - 0.01
    w0, w1, w2, w3, b0, b1, b2 = w
    m = oracle.Model(oracle.MLPNET, net=_net(w0, w1, w2, w3, b0, b1, b2, -0.5))
    if dead == 0:  # h1 = 0
        want = w3 @ (w2 @ b1 + b2) - 0.5
    elif dead == 1:  # h2 = 0
        want = w3 @ b2 - 0.5
    else:  # h3 = 0
        want = -0.5
    for _ in range(10):
        x = np.abs(rng.normal(0, 3, NIN))
        assert oracle.mlpnet_eval(m, x) == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_positive_homogeneity_without_biases():
    rng = np.random.default_rng(3)
    w0, w1, w2, w3, *_ = _rand(rng, pos=False)
    z = np.zeros(H)
    m = oracle.Model(oracle.MLPNET, net=_net(w0, w1, w2, w3, z, z, z, 0.0))
    for c in (0.5, 2.0, 7.0):
        x = rng.normal(0, 2, NIN)
        assert oracle.mlpnet_eval(m, c * x) == pytest.approx(c * oracle.mlpnet_eval(m, x), rel=1e-12, abs=1e-15)


def test_site_energy_of_a_pure_element():
    """Every site of species s: one-hot s, and 8, 6, 12 neighbours of s in
    shells 1, 2, 3."""
    net = inputs.mlpnet_weights(4)
    m = oracle.Model(oracle.MLPNET, net=net)
    S = 5
    lat = oracle.Lattice(4, 4, 4, S)
    for s in (0, 3):
        occ = np.full(lat.nsites, s, dtype=np.int8)
        x = np.zeros(NIN)
        x[s] = 1.0
        x[5 + s], x[10 + s], x[15 + s] = 8.0, 6.0, 12.0
        want = oracle.mlpnet_eval(m, x)
        assert oracle.total_energy(lat, m, occ) == pytest.approx(lat.nsites * want, rel=1e-12)


def test_delta_e_is_the_change_of_the_total():
    net = inputs.mlpnet_weights(5)
    m = oracle.Model(oracle.MLPNET, net=net)
    S = 5
    lat = oracle.Lattice(4, 5, 4, S)
    occ = oracle.init_lattice(lat, inputs.dirichlet_counts(lat.nsites, S, 2), 2)
    rng = np.random.default_rng(7)
    for _ in range(15):
        a = int(rng.integers(lat.nsites))
        b = oracle.neighbor(lat, a, oracle.shell_vectors(1)[rng.integers(8)])
        e0 = oracle.total_energy(lat, m, occ)
        d = oracle.delta_e(lat, m, occ, a, b)
        occ[a], occ[b] = occ[b], occ[a]
        assert d == pytest.approx(oracle.total_energy(lat, m, occ) - e0, abs=1e-10)
