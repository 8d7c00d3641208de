"""The slab mini-step on the GPU (Sec. III-B, 1D slab decomposition).

W slabs of one box are held as device windows in one process; every
mini-step runs slab by slab through smc_slab_ministep and is followed by the
ghost exchange as device-to-device copies (slab.LocalSlabExchange, the ranges
of slab.SlabPlan).  The assembled box must equal the unsharded smc_sweep bit
for bit, with the same accepted count (integer models: the same energy sum;
FP32: the same occupancy and count).  The split form -- the edge link cells
of every slab, the exchange, then the interior link cells, the order that
overlaps the transfer with the interior trials -- must give the same box."""
import numpy as np
import pytest

from paper_2604_08250_gb300 import inputs, slab

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


def dev():
    return torch.device("cuda:0")


def _run(smc, dims, S, nsh, W, nsweeps, order, is_int=True, seed=9):
    if is_int:
        model = smc.Model(smc.PAIR_I32, nsh, inputs.pair_int_coeffs(3, nsh, S), unit_ev=1e-4)
        kT = 0.03
    else:
        model = smc.Model(smc.PAIR_F32, nsh, inputs.pair_f32_coeffs(3, nsh, S))
        kT = 0.08
    lat = smc.Lattice(*dims, S)
    occ = torch.empty(lat.nsites, dtype=torch.int8, device=dev())
    smc.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, S), seed, occ)
    ref = occ.clone()
    e_ref = torch.zeros(1, dtype=torch.float64, device=dev())
    n_ref = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.sweep(lat, model, ref, seed, 0, nsweeps, kT, e_acc=e_ref, n_acc=n_ref)
    plan = slab.SlabPlan(*dims, W, 2)
    box0 = occ.cpu().numpy()
    wins = [torch.from_numpy(plan.window_of(box0, r)).to(dev()).contiguous() for r in range(W)]
    ex = slab.LocalSlabExchange(plan)
    e = torch.zeros(1, dtype=torch.float64, device=dev())
    n = torch.zeros(1, dtype=torch.int64, device=dev())

    def part(p, t, k):
        for r in range(W):
            smc.slab_ministep(lat, model, wins[r], plan.x0(r), plan.w, plan.ghost, seed, t, k, kT, part=p,
                              e_acc=e, n_acc=n)

    for t in range(nsweeps):
        for k in range(plan.nA):
            if order == "whole":
                part(0, t, k)
                ex.step(wins, t, k)
            else:
                part(1, t, k)
                ex.step(wins, t, k)
                part(2, t, k)
    smc.check()
    box = np.concatenate([plan.owned(w.cpu().numpy()) for w in wins], axis=-1).reshape(-1)
    assert np.array_equal(box, ref.cpu().numpy())
    for r in range(W):  # ghosts up to date too
        assert np.array_equal(wins[r].cpu().numpy(), plan.window_of(box, r))
    assert int(n.item()) == int(n_ref.item()) > 0
    if is_int:
        assert float(e.item()) == pytest.approx(float(e_ref.item()), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("dims,S,nsh,W", [((16, 8, 8), 3, 2, 2), ((32, 8, 12), 5, 2, 4), ((48, 12, 8), 4, 3, 3),
                                          ((16, 8, 8), 2, 2, 1), ((64, 8, 8), 5, 3, 2)])
@pytest.mark.parametrize("order", ["whole", "split"])
def test_slabs_equal_the_unsharded_sweep(smc, dims, S, nsh, W, order):
    _run(smc, dims, S, nsh, W, 2, order)


def test_slabs_equal_the_unsharded_sweep_fp32(smc):
    _run(smc, (32, 8, 8), 5, 2, 2, 2, "split", is_int=False)


def test_slab_ministep_rejects_bad_arguments(smc):
    lat = smc.Lattice(16, 8, 8, 3)
    model = smc.Model(smc.PAIR_I32, 2, inputs.pair_int_coeffs(3, 2, 3), unit_ev=1e-4)
    win = torch.zeros(2 * 8 * 8 * 12, dtype=torch.int8, device=dev())
    for x0, w, g, part in [(2, 8, 2, 0), (0, 8, 1, 0), (0, 6, 2, 0), (12, 8, 2, 0), (0, 8, 2, 3)]:
        with pytest.raises(smc.SMCError):
            smc.slab_ministep(lat, model, win, x0, w, g, 1, 0, 0, 0.03, part=part)
