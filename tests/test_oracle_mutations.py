"""Planted mistakes in the oracle: each one is a one-line change to
oracle/smc_oracle.c compiled into a temporary library, and at least one pin
must fail on it.  This checks that the pins test the oracle's arithmetic
(geometry, RNG, pair and qSRO energies and gradients, the zone of dE, the
network, the acceptance rule), not themselves.  The broken builds are loaded only inside these tests."""
import ctypes
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_energy as energy_pins
from tests import test_oracle_fcc as fcc_pins
from tests import test_oracle_geometry_rng as geo_pins
from tests import test_oracle_mc as mc_pins
from tests import test_oracle_mlpnet as net_pins
from tests import test_oracle_qsro as qsro_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "smc_oracle.c")

# name: ([(original line, planted line)], pins expected to fail)
MUTANTS = {
    "philox_multiplier": ([("#define PH_M0 0xD2511F53u", "#define PH_M0 0xD2511F55u")],
                          [geo_pins.test_philox_known_answers]),
    "pair_shells_reversed": ([("e2 += m->v_i32[((sh - 1) * S + occ[i]) * S + occ[j]];",
                               "e2 += m->v_i32[((m->nshells - sh) * S + occ[i]) * S + occ[j]];")],
                             [energy_pins.test_b2_ground_state_energy_closed_form]),
    "qsro_w_term_linear": ([("e += (double)m->qsro_w[(sh - 1) * S + p] * pi * pi;",
                             "e += (double)m->qsro_w[(sh - 1) * S + p] * pi;")],
                           [fcc_pins.test_qsro_l12_closed_form, lambda: qsro_pins.test_b2(2)]),
    "fcc_sublattices_exchanged": ([("case 5: nsub = 2; break;", "case 5: nsub = 3; break;"),
                                   ("case 3: nsub = 3; break;", "case 3: nsub = 2; break;")],
                                  [fcc_pins.test_shells_by_brute_force_distance]),
    "fcc_zone_without_b_side": ([("            om[n++] = orc_fcc_neighbor(lat, b, v[0], v[1], v[2]);\n", "")],
                                [lambda: fcc_pins.test_delta_e_is_the_change_of_the_total(2, "int"),
                                 lambda: fcc_pins.test_qsro_delta_e_is_the_change_of_the_total(2, (8, 8, 8))]),
    "mlpnet_second_relu_dropped": ([("        h2[k] = relu(z);", "        h2[k] = z;")],
                                   [lambda: net_pins.test_dead_layer_closed_forms(1)]),
    "metropolis_at_twice_the_temperature": ([("    return u < exp(-dE / kT);", "    return u < exp(-dE / (2.0 * kT));")],
                                            [qsro_pins.test_chain_matches_enumeration_16_site]),
    "integer_table_at_twice_the_temperature": ([("double t = floor(R_SCALE * exp(-(double)d * unit_ev / kT));",
                                                 "double t = floor(R_SCALE * exp(-(double)d * unit_ev / (2.0 * kT)));")],
                                               [lambda: mc_pins.test_boltzmann_enumeration_16_site(0.025)]),
    "bcc_neighbor_wraps_y_by_nx": ([("    int64_t cy = floor_mod((py - nsub) / 2, lat->ny);",
                                     "    int64_t cy = floor_mod((py - nsub) / 2, lat->nx);")],
                                   [lambda: geo_pins.test_neighbor_matches_bruteforce((4, 6, 8))]),
    "mlp_features_count_own_species": ([("            x[ORC_MLP_SPECIES * m + occ[j]] += 1.0;",
                                         "            x[ORC_MLP_SPECIES * m + occ[i]] += 1.0;")],
                                       [energy_pins.test_mlp_features_on_b2]),
    "qsro_linear_diagonal_doubled": ([("for (int r = 0; r <= p; ++r) e += (double)m->v_f32[((sh - 1) * S + p) * S + r] * (n[p][r] / total);",
                                       "for (int r = 0; r <= p; ++r) e += (double)m->v_f32[((sh - 1) * S + p) * S + r] * ((r == p ? 2.0 : 1.0) * n[p][r] / total);")],
                                     [lambda: qsro_pins.test_linear_sum_is_the_strict_form_reparametrised("fcc", 2, True),
                                      lambda: qsro_pins.test_linear_sum_is_the_strict_form_reparametrised("bcc", 1, False)]),
    "qsro_gradient_of_w_linear": ([("                gW[(sh - 1) * S + p] += pi * pi;",
                                    "                gW[(sh - 1) * S + p] += pi;")],
                                  [qsro_pins.test_gradient_equals_finite_differences]),
}


def _build_mutant(name, edits, tmp):
    src = open(SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    c_path = os.path.join(tmp, f"{name}.c")
    so_path = os.path.join(tmp, f"lib{name}.so")
    with open(c_path, "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-I",
                    os.path.dirname(SRC), "-o", so_path, c_path, "-lm"], check=True)
    return oracle.bind(ctypes.CDLL(so_path))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path, monkeypatch):
    edits, pins = MUTANTS[name]
    # the pins hold on the real oracle
    for pin in pins:
        pin()
    monkeypatch.setattr(oracle, "_lib", _build_mutant(name, edits, str(tmp_path)))
    failed = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1, f"no pin caught the planted mistake {name}"
