"""Batched replicas of uneven sizes on a temperature ladder: the autotuner
(timing candidate tile shapes and CTA sizes on copies) and a CUDA-graph
capture of one multi-sweep batched call.  The replayed graph, run with the
tuning the autotuner picked, must give the occupancies and accepted counts
of direct calls with the library's default tuning bit for bit (the tuning
changes no result); e_acc is summed per tile, so its rounding may differ
with the tile shape."""
import numpy as np
import pytest

from paper_2604_08250_gb300 import inputs

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


def test_autotuned_graph_replay_equals_direct_calls(smc):
    from paper_2604_08250_gb300 import autotune
    S, seed, nsw = 5, 13, 6
    model = smc.Model(smc.PAIR_F32, 2, inputs.pair_f32_coeffs(3, 2, S))
    edges = [32, 40, 48, 16]
    lats = [smc.Lattice(e, e, e, S) for e in edges]
    occs = []
    for r, l in enumerate(lats):
        o = torch.empty(l.nsites, dtype=torch.int8, device="cuda")
        smc.init_lattice(l, inputs.equiatomic_counts(l.nsites, S), seed, o, replica=r)
        occs.append(o)
    kT = inputs.ladder_kT(len(lats), 300.0, 3000.0)
    kTb = np.repeat(kT[:, None], nsw, axis=1)
    start = [o.clone() for o in occs]
    # direct calls, default tuning
    smc.set_tuning()
    ref = [o.clone() for o in occs]
    e_ref = torch.zeros(len(lats), dtype=torch.float64, device="cuda")
    n_ref = torch.zeros(len(lats), dtype=torch.int64, device="cuda")
    smc.sweep_batched(lats, model, ref, seed, 0, nsw // 2, kTb[:, : nsw // 2], e_acc=e_ref, n_acc=n_ref)
    smc.sweep_batched(lats, model, ref, seed, nsw // 2, nsw // 2, kTb[:, nsw // 2:], e_acc=e_ref, n_acc=n_ref)
    smc.check()
    try:
        best, times = autotune.autotune_batched(lats, model, occs, seed, kT)
        assert best in times and len(times) >= 4
        assert all(torch.equal(o, s0) for o, s0 in zip(occs, start))  # tuned on copies
        e_acc = torch.zeros(len(lats), dtype=torch.float64, device="cuda")
        n_acc = torch.zeros(len(lats), dtype=torch.int64, device="cuda")
        g = autotune.capture_batched(lats, model, occs, seed, 0, nsw, kTb, e_acc=e_acc, n_acc=n_acc)
        assert all(torch.equal(o, s0) for o, s0 in zip(occs, start))  # capture runs nothing
        assert int(n_acc.sum().item()) == 0
        g.replay()
        torch.cuda.synchronize()
        smc.check()
        for o, r in zip(occs, ref):
            assert torch.equal(o, r)
        assert torch.equal(n_acc, n_ref)
        assert torch.allclose(e_acc, e_ref, rtol=1e-9, atol=1e-9)
    finally:
        smc.set_tuning()
