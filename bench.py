"""Benchmark: Metropolis swap attempts/s on one GB300 (and N independent
replicas under torchrun).

Workload (one "step" = one full job of the config-2 workload): a BCC box of
128^3 cells (4,194,304 sites), five species at equal counts, FP32 pair
coefficients over two shells drawn N(0, 20 meV), annealed linearly from 3000 K
to 300 K over 1000 sweeps (one trial per site per sweep), followed by the
total energy and the Warren-Cowley SRO of shells 1-3.  Inputs are synthetic and
resident in device memory when the timed region starts; L2 is flushed between
steps.  Extra lines of the JSON object report the 512^3 HBM-resident case,
the batched replica ladder and the energy gradient against the plain sweep.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_08250_gb300 import inputs, replicas  # noqa: E402

METRIC = "MC swap attempts/s on 1 GB300 (% HBM roofline); batched & grad vs plain sweep"
BYTES_PER_ATTEMPT = 24.0  # 22 B read set + 2 B written per trial (two-shell pair model)
# MLP 20-64-64-1: dense products per site evaluation, forward only and forward + backward
# MLPNet (20 -> 96 -> 96 -> 96 -> 1): 2 (20 96 + 96 96 + 96 96 + 96) FLOP per
# site evaluation, 40 post-swap evaluations per attempt (pre-swap energies cached)
NET_FLOP_PER_SITE = 2 * (20 * 96 + 96 * 96 + 96 * 96 + 96)
NET_FLOP_PER_ATTEMPT = 40 * NET_FLOP_PER_SITE
QSRO_SEED, QSRO_SHELLS = 7, 2  # qSRO workload parameters
# zone sites of a qSRO trial besides a and b (within the model's shells of
# either), counted from the BCC geometry
QSRO_ZONE = {1: 14, 2: 20, 3: 38}
MLP_FLOP_PER_SITE_FWD = 2 * (20 * 64 + 64 * 64)  # 10752
MLP_FLOP_PER_SITE_GRAD = MLP_FLOP_PER_SITE_FWD + 2 * 64 * 64 + 2 * 64 * 64 + 2 * 20 * 64  # 29696
MLP_FLOP_PER_ATTEMPT = 40 * MLP_FLOP_PER_SITE_FWD  # post-swap energies of the 40-site zone (cached pre-swap)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def config2_problem():
    c = inputs.CONFIG2
    dims, S = c["cells"], c["nspecies"]
    N = 2 * dims[0] * dims[1] * dims[2]
    return dict(dims=dims, S=S, N=N, V=inputs.pair_f32_coeffs(c["coeff_seed"], 2, S),
                counts=inputs.equiatomic_counts(N, S), kT=inputs.anneal_kT(c["nsweeps"], c["t_start"], c["t_end"]),
                nsweeps=c["nsweeps"], seed=c["mc_seed"])


def cpu_baseline(prob, mini_steps: int):
    """The oracle as it stands, serial, on the first `mini_steps` mini-steps of
    sweep 0 of the config-2 lattice (32,768 trials each)."""
    import oracle
    lat = oracle.Lattice(*prob["dims"], prob["S"])
    model = oracle.Model(oracle.PAIR_F32, 2, prob["V"])
    occ = oracle.init_lattice(lat, prob["counts"], prob["seed"])
    nA, _ = oracle.schedule(lat)
    t0 = time.perf_counter()
    ntr = 0
    for k in range(mini_steps):
        dE, _, _, _ = oracle.ministep_trace(lat, model, occ, prob["seed"], 0, k, float(prob["kT"][0]))
        ntr += len(dE)
    dt = time.perf_counter() - t0
    return ntr / dt, ntr, dt


def cpu_baseline_qsro(mini_steps: int):
    """The oracle on the qSRO workload's model and composition: the first
    `mini_steps` mini-steps of sweep 0 of a 128^3 box (32,768 trials each)."""
    import oracle
    c4 = inputs.CONFIG4
    S = c4["nspecies"]
    V, W, C = inputs.qsro_coeffs(QSRO_SEED, QSRO_SHELLS, S)
    lat = oracle.Lattice(128, 128, 128, S)
    model = oracle.Model(oracle.QSRO, QSRO_SHELLS, V, qsro_w=W, qsro_c=C)
    occ = oracle.init_lattice(lat, inputs.dirichlet_counts(lat.nsites, S, c4["comp_seed"]), c4["mc_seed"])
    t0 = time.perf_counter()
    ntr = 0
    for k in range(mini_steps):
        dE, _, _, _ = oracle.ministep_trace(lat, model, occ, c4["mc_seed"], 0, k, inputs.K_B_EV * c4["T"])
        ntr += len(dE)
    dt = time.perf_counter() - t0
    return ntr / dt, ntr, dt


def run_reference(args, rank):
    """Reference arm: the serial CPU oracle on the same workload and metric,
    a bounded sample of the job per step."""
    if rank != 0:
        return
    prob = config2_problem()
    per_step = 8  # mini-steps of sweep 0 per step (262,144 trials)
    for _ in range(args.warmup):
        cpu_baseline(prob, 1)
    tot_tr, tot_t = 0, 0.0
    for _ in range(args.steps):
        rate, ntr, dt = cpu_baseline(prob, per_step)
        tot_tr += ntr
        tot_t += dt
    v = tot_tr / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "attempts/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "bcc128_quinary_f32_pair_anneal", "cells": [128, 128, 128], "sites": prob["N"],
                       "sample": f"{per_step} mini-steps of sweep 0 per step"},
            "cpu_baseline": {"value": v, "unit": "attempts/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} mini-steps (x32768 trials) of sweep 0 per step, serial C"},
            "e2e": {"value": v, "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the 512^3, batched and gradient lines")
    ap.add_argument("--cpu-mini-steps", type=int, default=24)
    ap.add_argument("--profile-sweep", type=int, default=0,
                    help="profiling driver: one sweep launch on an N^3 quinary FP32 lattice, nothing else")
    ap.add_argument("--profile-sweeps", type=int, default=1)
    ap.add_argument("--profile-counts", type=int, default=0,
                    help="profiling driver: the pair gradient (bit planes + pair counts) of an N^3 quinary lattice")
    ap.add_argument("--profile-mlp", type=int, default=0,
                    help="run the MLP workload (800 K) on a 256 x n x n box once, for ncu captures")
    ap.add_argument("--profile-mlpnet", type=int, default=0,
                    help="as --profile-mlp, with MLPNet at the paper's shape")
    ap.add_argument("--profile-qsro", type=int, default=0,
                    help="run the qSRO workload (800 K) on an N^3 box once, for ncu captures")
    ap.add_argument("--profile-fcc", type=int, default=0,
                    help="run FCC sweeps (800 K) on an N^3 box of cubic cells once, for ncu captures")
    ap.add_argument("--profile-fcc-qsro", type=int, default=0,
                    help="as --profile-fcc with the qSRO workload (Fe29Co29Ni28Al7Ti7, 2 shells)")
    args = ap.parse_args()
    if args.profile_fcc:
        profile_fcc(args.profile_fcc, args.profile_sweeps)
        return
    if args.profile_fcc_qsro:
        profile_fcc(args.profile_fcc_qsro, args.profile_sweeps, qsro=True)
        return
    if args.profile_mlp:
        profile_mlp(args.profile_mlp, args.profile_sweeps)
        return
    if args.profile_mlpnet:
        profile_mlp(args.profile_mlpnet, args.profile_sweeps, net=True)
        return
    if args.profile_qsro:
        profile_qsro(args.profile_qsro, args.profile_sweeps)
        return
    if args.profile_sweep:
        profile_sweep(args.profile_sweep, args.profile_sweeps)
        return
    if args.profile_counts:
        profile_counts(args.profile_counts)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    from paper_2604_08250_gb300 import build as _b
    from paper_2604_08250_gb300 import smc
    _b.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    pk = peaks()
    prob = config2_problem()
    lat = smc.Lattice(*prob["dims"], prob["S"])
    model = smc.Model(smc.PAIR_F32, 2, prob["V"])
    occ0 = torch.empty(prob["N"], dtype=torch.int8, device=dev)
    smc.init_lattice(lat, prob["counts"], prob["seed"], occ0, replica=rank)
    occ = torch.empty_like(occ0)
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev)
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev)
    energy = torch.zeros(1, dtype=torch.float64, device=dev)
    counts = torch.zeros((3, prob["S"], prob["S"]), dtype=torch.int64, device=dev)
    alpha = torch.zeros((3, prob["S"], prob["S"]), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()
    nsw = prob["nsweeps"]
    # our kernels per step: lattice copy + resident sweep; bit planes + pair
    # counts + energy finish; bit planes + pair counts + SRO finish
    launches_per_step = 2 + 3 + 3

    def job(sw_ev=None):
        if sw_ev:
            sw_ev[0].record(stream)
        smc.sweep(lat, model, occ, prob["seed"], 0, nsw, prob["kT"], replica=rank, e_acc=e_acc, n_acc=n_acc)
        if sw_ev:
            sw_ev[1].record(stream)
        smc.energy(lat, model, occ, e=energy)
        smc.sro(lat, 3, occ, counts=counts, alpha=alpha)

    for _ in range(args.warmup):
        occ.copy_(occ0)
        job()
    smc.check()

    step_ms, sweep_ms = [], []
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            occ.copy_(occ0)
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            s0, s1 = torch.cuda.Event(True), torch.cuda.Event(True)
            e0.record(stream)
            job((s0, s1))
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            sweep_ms.append(s0.elapsed_time(s1))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    smc.check()
    attempts_step = prob["N"] * nsw
    value, total_ms = replicas.job_throughput(float(sum(step_ms)), attempts_step * args.steps, dist, dev)
    sweep_launch_s = float(np.mean(sweep_ms)) * 1e-3
    achieved = BYTES_PER_ATTEMPT * attempts_step / sweep_launch_s / 1e9

    # ---- end to end through the C ABI with host buffers ----
    host_occ = torch.empty(prob["N"], dtype=torch.int8, pin_memory=True)
    host_occ.copy_(occ0.cpu())
    host_out = torch.empty(prob["N"], dtype=torch.int8, pin_memory=True)
    host_obs = torch.empty(1 + 2 * 3 * prob["S"] * prob["S"], dtype=torch.float64, pin_memory=True)
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        occ.copy_(host_occ, non_blocking=True)
        job()
        host_out.copy_(occ, non_blocking=True)
        host_obs[0:1].copy_(energy, non_blocking=True)
        host_obs[1:1 + counts.numel()].copy_(counts.reshape(-1).double(), non_blocking=True)
        host_obs[1 + counts.numel():].copy_(alpha.reshape(-1), non_blocking=True)
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_value, _ = replicas.job_throughput(float(sum(e2e_ms)), attempts_step * args.steps, dist, dev)

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(smc, torch, dev, pk)
    cpu = None
    if rank == 0:
        rate, ntr, dt = cpu_baseline(prob, args.cpu_mini_steps)
        cpu = {"value": rate, "unit": "attempts/s", "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_mini_steps} mini-steps (x32768 trials) of sweep 0 of the 128^3 job, "
                         f"serial C oracle, {dt:.1f} s"}
        if extras:
            qrate, qntr, qdt = cpu_baseline_qsro(2)
            cpu["qsro"] = {"value": qrate, "unit": "attempts/s", "cores": 1, "kind": "oracle",
                           "sample": f"2 mini-steps (x32768 trials) of the qSRO workload's model on a 128^3 box, "
                                     f"serial C oracle, {qdt:.1f} s"}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    traffic = profile_record("k_sweep_resident_bcc128_1000sweeps", "bytes_per_launch")
    line = {
        "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded draws; BCC, 5 species, FP32 pair model)",
        "config": {"workload": "bcc128_quinary_f32_pair_anneal", "cells": [128, 128, 128], "sites": prob["N"],
                   "sweeps_per_step": nsw, "attempts_per_step": attempts_step, "species": prob["S"], "shells": 2,
                   "anneal_K": [3000, 300], "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                     "kernel": "k_sweep_resident (one launch = 1000 sweeps)",
                     "bytes_per_attempt": BYTES_PER_ATTEMPT, "peak_source": pk["source"] + " hbm_gbs",
                     "note": "the 4.2 MB lattice stays in shared memory for the launch; see extras.hbm_512 "
                             "for the HBM-resident case"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "attempts/s", "h2d_bytes_per_step": prob["N"],
                "d2h_bytes_per_step": prob["N"] + 8 * (1 + 2 * 3 * prob["S"] * prob["S"])},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
        "extras": extras,
    }
    print(json.dumps(line), flush=True)


def profile_sweep(n: int, nsweeps: int):
    """Runs exactly one sweep launch (nsweeps sweeps) of the n^3 config-2
    model after initialisation, for ncu captures (-k regex:k_sweep)."""
    import torch
    from paper_2604_08250_gb300 import build as _b
    from paper_2604_08250_gb300 import smc
    _b.build()
    smc.debug_set(smc.DBG_TIMEOUT_MS, 60000)  # replayed launches run slower under the profiler
    S = 5
    lat = smc.Lattice(n, n, n, S)
    occ = torch.empty(lat.nsites, dtype=torch.int8, device="cuda")
    smc.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, S), 1, occ)
    model = smc.Model(smc.PAIR_F32, 2, inputs.pair_f32_coeffs(inputs.CONFIG2["coeff_seed"], 2, S))
    smc.sweep(lat, model, occ, 1, 0, nsweeps, inputs.anneal_kT(1000)[:nsweeps])
    smc.check()
    print(json.dumps({"profile_sweep": n, "sweeps": nsweeps, "ok": True}))


def profile_counts(n: int):
    """One pair-gradient call (bit planes, pair counts, finish) on the n^3
    config-2 lattice, for ncu captures (-k regex:k_pair_counts)."""
    import torch
    from paper_2604_08250_gb300 import build as _b
    from paper_2604_08250_gb300 import smc
    _b.build()
    S = 5
    lat = smc.Lattice(n, n, n, S)
    occ = torch.empty(lat.nsites, dtype=torch.int8, device="cuda")
    smc.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, S), 1, occ)
    model = smc.Model(smc.PAIR_F32, 2, inputs.pair_f32_coeffs(inputs.CONFIG2["coeff_seed"], 2, S))
    g = torch.zeros(smc.grad_size(lat, model), dtype=torch.float32, device="cuda")
    smc.energy_grad(lat, model, occ, g)
    smc.check()
    print(json.dumps({"profile_counts": n, "ok": True}))


def qsro_setup(smc, n: int, dev):
    """qSRO workload: N^3 cells, the MLP workload's Dirichlet quinary
    composition, 2-shell qSRO parameters (seed 7), 800 K."""
    c4 = inputs.CONFIG4
    S = c4["nspecies"]
    V, W, C = inputs.qsro_coeffs(QSRO_SEED, QSRO_SHELLS, S)
    model = smc.Model(smc.QSRO_F32, QSRO_SHELLS, V, qsro_w=W, qsro_c=C)
    import torch
    lat = smc.Lattice(n, n, n, S)
    occ = torch.empty(lat.nsites, dtype=torch.int8, device=dev)
    smc.init_lattice(lat, inputs.dirichlet_counts(lat.nsites, S, c4["comp_seed"]), c4["mc_seed"], occ)
    return lat, occ, model, inputs.K_B_EV * c4["T"]


def fcc_setup(smc, n: int, dev, qsro: bool = False):
    """FCC workloads, N^3 cubic cells (4 N^3 sites), 800 K, the first two
    shells (12 + 6 neighbours): equiatomic quinary with FP32 pair
    coefficients (seed 3); or (qsro) the paper's Fe29Co29Ni28Al7Ti7 with
    qSRO parameters (seed 7)."""
    import torch
    S = 5
    lat = smc.Lattice(n, n, n, S)
    N = smc.fcc_nsites(lat)
    occ = torch.empty(N, dtype=torch.int8, device=dev)
    if qsro:
        smc.fcc_init_lattice(lat, inputs.fraction_counts(N, inputs.HEA_FRACTIONS), 1, occ)
        V, W, C = inputs.qsro_coeffs(QSRO_SEED, 2, S)
        model = smc.Model(smc.QSRO_F32, 2, V, qsro_w=W, qsro_c=C)
    else:
        smc.fcc_init_lattice(lat, inputs.equiatomic_counts(N, S), 1, occ)
        model = smc.Model(smc.PAIR_F32, 2, inputs.pair_f32_coeffs(3, 2, S))
    return lat, occ, model, inputs.K_B_EV * 800.0


def profile_fcc(n: int, nsweeps: int, qsro: bool = False):
    """FCC sweeps on an N^3 box, for ncu captures (-k regex:k_fcc_)."""
    from paper_2604_08250_gb300 import build as _b
    from paper_2604_08250_gb300 import smc
    _b.build()
    lat, occ, model, kT = fcc_setup(smc, n, "cuda", qsro=qsro)
    smc.fcc_sweep(lat, model, occ, 1, 0, nsweeps, kT)
    smc.check()
    del occ
    print(json.dumps({"profile_fcc": n, "qsro": qsro, "sweeps": nsweeps, "ok": True}))


def profile_qsro(n: int, nsweeps: int):
    """qSRO sweeps on an N^3 box (the count-cache kernel k_bq_cache, then 128
    mini-step launches of k_bq_ministep per sweep), for ncu captures."""
    import torch
    from paper_2604_08250_gb300 import build as _b
    from paper_2604_08250_gb300 import smc
    _b.build()
    smc.debug_set(smc.DBG_TIMEOUT_MS, 60000)  # replayed launches run slower under the profiler
    lat, occ, model, kT = qsro_setup(smc, n, "cuda")
    smc.sweep(lat, model, occ, inputs.CONFIG4["mc_seed"], 0, nsweeps, kT)
    smc.check()
    del occ
    torch.cuda.synchronize()
    print(json.dumps({"profile_qsro": n, "sweeps": nsweeps, "ok": True}))


def profile_mlp(n: int, nsweeps: int, net: bool = False):
    """One MLP sweep launch (nsweeps sweeps; the energy-cache kernel runs
    first) and one energy evaluation on a 256 x n x n box with the MLP
    workload's composition, weights and temperature, for ncu captures
    (-k regex:k_sweep_mlp or regex:k_mlp_site_energy); net: MLPNet at the
    paper's shape instead of the 64-wide network."""
    import torch
    from paper_2604_08250_gb300 import build as _b
    from paper_2604_08250_gb300 import smc
    _b.build()
    smc.debug_set(smc.DBG_TIMEOUT_MS, 60000)  # replayed launches run slower under the profiler
    c4 = inputs.CONFIG4
    S = c4["nspecies"]
    lat = smc.Lattice(256, n, n, S)
    occ = torch.empty(lat.nsites, dtype=torch.int8, device="cuda")
    smc.init_lattice(lat, inputs.dirichlet_counts(lat.nsites, S, c4["comp_seed"]), c4["mc_seed"], occ)
    if net:
        model = smc.Model(smc.MLPNET_BF16, net=inputs.mlpnet_weights(c4["mlp_seed"]))
    else:
        model = smc.Model(smc.MLP_BF16, mlp=inputs.mlp_weights(c4["mlp_seed"]))
    smc.sweep(lat, model, occ, c4["mc_seed"], 0, nsweeps, inputs.K_B_EV * c4["T"])
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    smc.energy(lat, model, occ, e)
    smc.check()
    print(json.dumps({"profile_mlp": [256, n, n], "net": net, "sweeps": nsweeps, "ok": True}))


def profile_record(name: str, field: str):
    """A counter figure from profiles/traffic.json (ncu, per launch), or None
    when a source it names changed after the counters were taken."""
    import hashlib
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tp):
        return None
    with open(tp) as f:
        d = json.load(f).get(name)
    if not d or field not in d:
        return None
    for src, sha in d["sources"].items():
        with open(os.path.join(ROOT, src), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != sha:
                return None
    return d[field]


def run_extras(smc, torch, dev, pk):
    out = {}
    stream = torch.cuda.current_stream()
    S = 5
    V = inputs.pair_f32_coeffs(inputs.CONFIG2["coeff_seed"], 2, S)
    model = smc.Model(smc.PAIR_F32, 2, V)

    def unlike_fraction(l, o):
        # fraction of first-shell bonds joining two species: the share of
        # attempts (partner = a first-shell neighbour) the MLP sweeps evaluate
        c = torch.zeros((1, S, S), dtype=torch.int64, device=dev)
        smc.sro(l, 1, o, counts=c)
        c = c[0].double()
        return float(1.0 - torch.diagonal(c).sum() / c.sum())

    def timed(fn, reps=1):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps

    # 512^3: lattice (268 MB) larger than L2 -> HBM-resident
    n = 512
    lat = smc.Lattice(n, n, n, S)
    occ = torch.empty(lat.nsites, dtype=torch.int8, device=dev)
    smc.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, S), 1, occ)
    kT = inputs.anneal_kT(1000)
    nsw = 20
    ms = timed(lambda: smc.sweep(lat, model, occ, 1, 0, nsw, kT[:nsw]), reps=2)
    att = lat.nsites * nsw / (ms * 1e-3)
    out["hbm_512"] = {"cells": [n, n, n], "sweeps_per_launch": nsw, "ms_per_sweep": ms / nsw,
                      "attempts_per_s": att, "achieved_gbs": att * BYTES_PER_ATTEMPT / 1e9,
                      "frac_of_measured_hbm": att * BYTES_PER_ATTEMPT / 1e9 / pk["hbm_gbs"],
                      "kernel": "k_sweep_pairs (groups in pairs; the call includes the species scaling "
                                "passes around the launch)",
                      "dram_bytes_per_attempt": profile_record("k_sweep_pairs_bcc512_4sweeps", "bytes_per_attempt")}
    # integer-issue ceiling beside the HBM one: every SM issues at most 4 warp
    # instructions (128 lanes) per clock, and a trial costs the instructions
    # ncu counted on this kernel source (None once the source changed)
    ipt = profile_record("k_sweep_pairs_bcc512_4sweeps", "instructions_per_trial")
    if ipt:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        issue_cap = sms * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6 / ipt
        out["hbm_512"]["alu"] = {"instructions_per_trial": ipt, "issue_ceiling_attempts_per_s": issue_cap,
                                 "frac_of_issue_ceiling": att / issue_cap,
                                 "source": "profiles/traffic.json: ncu smsp__inst_executed.sum x 32 / trials"}
    # gradient of E (pair part) at the 512^3 configuration vs one plain sweep of it
    g = torch.zeros(smc.grad_size(lat, model), dtype=torch.float32, device=dev)
    gms = timed(lambda: smc.energy_grad(lat, model, occ, g), reps=3)
    out["grad_512"] = {"ms_per_configuration": gms, "ms_per_plain_sweep": ms / nsw,
                       "ratio_to_sweep": gms / (ms / nsw), "params": int(g.numel()),
                       "bytes_per_site": 1, "achieved_gbs": lat.nsites / (gms * 1e-3) / 1e9,
                       "frac_of_measured_hbm": lat.nsites / (gms * 1e-3) / 1e9 / pk["hbm_gbs"]}
    del occ
    # batched: 64 uneven replicas on a temperature ladder, one launch
    c3 = inputs.CONFIG3
    edges = inputs.batched_edges(c3["edge_seed"], c3["nrep"])
    lats = [smc.Lattice(int(e), int(e), int(e), S) for e in edges]
    occs = []
    for r, l in enumerate(lats):
        o = torch.empty(l.nsites, dtype=torch.int8, device=dev)
        smc.init_lattice(l, inputs.equiatomic_counts(l.nsites, S), 1, o, replica=r)
        occs.append(o)
    kTr = inputs.ladder_kT(c3["nrep"], c3["t_min"], c3["t_max"])
    # tile shape and CTA size picked by the autotuner (on copies of the
    # replicas), then all of the run's sweeps as one captured graph launch
    from paper_2604_08250_gb300 import autotune
    best, tune_ms = autotune.autotune_batched(lats, model, occs, 1, kTr, sweeps=2)
    nb = c3["nsweeps"]
    kTb = np.repeat(kTr[:, None], nb, axis=1)
    graph = autotune.capture_batched(lats, model, occs, 1, 0, nb, kTb)
    bms = timed(graph.replay, reps=1)
    smc.set_tuning()
    tot = sum(l.nsites for l in lats)
    batt = tot * nb / (bms * 1e-3)
    del graph
    for o in occs:
        del o
    occs.clear()
    # the matched plain sweep: one 256^3 lattice (3.4e7 sites, about the
    # ladder's 3.9e7), same model, one launch of the same number of sweeps at
    # the ladder's middle temperature
    n2 = 256
    lat2 = smc.Lattice(n2, n2, n2, S)
    occ2 = torch.empty(lat2.nsites, dtype=torch.int8, device=dev)
    smc.init_lattice(lat2, inputs.equiatomic_counts(lat2.nsites, S), 1, occ2)
    kTm = float(np.median(kTr))
    pms = timed(lambda: smc.sweep(lat2, model, occ2, 1, 0, nb, kTm), reps=1)
    patt = lat2.nsites * nb / (pms * 1e-3)
    del occ2
    out["batched_64"] = {"replicas": len(lats), "edges_min_max": [int(edges.min()), int(edges.max())],
                         "total_sites": tot, "sweeps": nb, "launch": "one CUDA graph replay (one persistent kernel)",
                         "tuning": {"tile_y": best[0], "tile_z": best[1], "threads": best[2], "ctas_per_sm": best[3]},
                         "tuning_ms_per_sweep": {"x".join(map(str, k)): round(v, 4) for k, v in tune_ms.items()},
                         "attempts_per_s": batt,
                         "frac_of_measured_hbm": batt * BYTES_PER_ATTEMPT / 1e9 / pk["hbm_gbs"],
                         "plain_sweep": {"cells": [n2] * 3, "sites": lat2.nsites, "sweeps": nb, "kT_eV": kTm,
                                         "attempts_per_s": patt},
                         "ratio_to_plain_sweep": batt / patt}
    # MLP site energies on the tensor cores: 256^3 Dirichlet quinary at 800 K
    c4 = inputs.CONFIG4
    n4 = c4["cells"][0]
    lat4 = smc.Lattice(n4, n4, n4, S)
    occ4 = torch.empty(lat4.nsites, dtype=torch.int8, device=dev)
    smc.init_lattice(lat4, inputs.dirichlet_counts(lat4.nsites, S, c4["comp_seed"]), c4["mc_seed"], occ4)
    mlp_model = smc.Model(smc.MLP_BF16, mlp=inputs.mlp_weights(c4["mlp_seed"]))
    kT4 = inputs.K_B_EV * c4["T"]
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev)
    nsw4 = 2
    f0 = unlike_fraction(lat4, occ4)
    ms4 = timed(lambda: smc.sweep(lat4, mlp_model, occ4, c4["mc_seed"], 0, nsw4, kT4, n_acc=n_acc), reps=1)
    fev = 0.5 * (f0 + unlike_fraction(lat4, occ4))
    att4 = lat4.nsites * nsw4 / (ms4 * 1e-3)
    acc_rate = float(n_acc.item()) / (2 * lat4.nsites * nsw4)  # warm-up call + timed call
    tfl = att4 * fev * MLP_FLOP_PER_ATTEMPT / 1e12
    out["mlp_256"] = {"cells": [n4] * 3, "sweeps_per_launch": nsw4, "ms_per_sweep": ms4 / nsw4,
                      "attempts_per_s": att4, "job_s_200_sweeps": ms4 / nsw4 * c4["nsweeps"] / 1e3,
                      "accept_rate": acc_rate, "evaluated_fraction": fev, "achieved_tflops": tfl,
                      "achieved_tflops_if_every_attempt": att4 * MLP_FLOP_PER_ATTEMPT / 1e12,
                      "frac_of_measured_bf16_sustained": tfl / pk["bf16_tflops_sustained"],
                      "flop_per_evaluated_attempt": MLP_FLOP_PER_ATTEMPT,
                      "note": "attempts with equal species (dE = 0) are not evaluated; evaluated_fraction is the "
                              "unlike first-shell bond fraction before and after the timed sweeps"}
    e4 = torch.zeros(1, dtype=torch.float64, device=dev)
    ems = timed(lambda: smc.energy(lat4, mlp_model, occ4, e4), reps=3)
    out["mlp_energy_256"] = {"ms": ems, "achieved_tflops": lat4.nsites * MLP_FLOP_PER_SITE_FWD / (ems * 1e-3) / 1e12}
    # MLPNet at the paper's shape on the same lattice and temperature
    net_model = smc.Model(smc.MLPNET_BF16, net=inputs.mlpnet_weights(c4["mlp_seed"]))
    n_accn = torch.zeros(1, dtype=torch.int64, device=dev)
    f0 = unlike_fraction(lat4, occ4)
    msn = timed(lambda: smc.sweep(lat4, net_model, occ4, c4["mc_seed"], 0, nsw4, kT4, n_acc=n_accn), reps=1)
    fevn = 0.5 * (f0 + unlike_fraction(lat4, occ4))
    attn = lat4.nsites * nsw4 / (msn * 1e-3)
    tfn = attn * fevn * NET_FLOP_PER_ATTEMPT / 1e12
    out["mlpnet_256"] = {"cells": [n4] * 3, "sweeps_per_launch": nsw4, "ms_per_sweep": msn / nsw4,
                         "attempts_per_s": attn, "accept_rate": float(n_accn.item()) / (2 * lat4.nsites * nsw4),
                         "evaluated_fraction": fevn, "achieved_tflops": tfn,
                         "achieved_tflops_if_every_attempt": attn * NET_FLOP_PER_ATTEMPT / 1e12,
                         "frac_of_measured_bf16_sustained": tfn / pk["bf16_tflops_sustained"],
                         "flop_per_evaluated_attempt": NET_FLOP_PER_ATTEMPT}
    en = torch.zeros(1, dtype=torch.float64, device=dev)
    emsn = timed(lambda: smc.energy(lat4, net_model, occ4, en), reps=3)
    out["mlpnet_energy_256"] = {"ms": emsn,
                                "achieved_tflops": lat4.nsites * NET_FLOP_PER_SITE / (emsn * 1e-3) / 1e12}
    del occ4
    # qSRO site energies (Eq. quadratic_local_SRO) on the cached-feature sweep, 256^3 at 800 K
    latq, occq, qm, kTq = qsro_setup(smc, 256, dev)
    nq = torch.zeros(1, dtype=torch.int64, device=dev)
    nswq = 4
    msq = timed(lambda: smc.sweep(latq, qm, occq, 1, 0, nswq, kTq, n_acc=nq), reps=1)
    attq = latq.nsites * nswq / (msq * 1e-3)
    accq = float(nq.item()) / (2 * latq.nsites * nswq)
    # bytes the design moves per attempt: species of a, b and the zone and the
    # zone's count-cache entries read (1 B each for 2 shells); when accepted the
    # two species and the cache entries of a, b and the zone written
    zq = QSRO_ZONE[QSRO_SHELLS]
    bq = 2 + 2 * zq + accq * (2 + 2 + zq)
    out["qsro_256"] = {"cells": [256] * 3, "shells": QSRO_SHELLS, "sweeps_per_launch": nswq,
                       "launches_per_sweep": 128, "ms_per_sweep": msq / nswq, "attempts_per_s": attq,
                       "accept_rate": accq, "bytes_per_attempt": bq, "achieved_gbs": attq * bq / 1e9,
                       "note": "67 MB of species and count cache: L2-resident, bound by load latency"}
    eq = torch.zeros(1, dtype=torch.float64, device=dev)
    emsq = timed(lambda: smc.energy(latq, qm, occq, eq), reps=3)
    out["qsro_energy_256"] = {"ms": emsq}
    del occq
    # FCC lattice (Sec. IV-C), FP32 2-shell quinary pair model, 256^3 cubic cells, 800 K
    latf, occf, fm, kTf = fcc_setup(smc, 256, dev)
    nf = torch.zeros(1, dtype=torch.int64, device=dev)
    nswf = 2
    msf = timed(lambda: smc.fcc_sweep(latf, fm, occf, 1, 0, nswf, kTf, n_acc=nf), reps=1)
    Nf = smc.fcc_nsites(latf)
    out["fcc_256"] = {"cells": [256] * 3, "sites": Nf, "shells": 2, "sweeps_per_launch": nswf,
                      "launches_per_sweep": 256, "ms_per_sweep": msf / nswf,
                      "attempts_per_s": Nf * nswf / (msf * 1e-3),
                      "accept_rate": float(nf.item()) / (2 * Nf * nswf)}
    ef = torch.zeros(1, dtype=torch.float64, device=dev)
    out["fcc_energy_256"] = {"ms": timed(lambda: smc.fcc_energy(latf, fm, occf, ef), reps=3)}
    del occf
    # the paper's workload shape: qSRO on the FCC lattice, Fe29Co29Ni28Al7Ti7, 2 shells, 256^3 cells, 800 K
    latq, occq, qm, kTq = fcc_setup(smc, 256, dev, qsro=True)
    nq = torch.zeros(1, dtype=torch.int64, device=dev)
    nswq = 2
    msq = timed(lambda: smc.fcc_sweep(latq, qm, occq, 1, 0, nswq, kTq, n_acc=nq), reps=1)
    Nq = smc.fcc_nsites(latq)
    out["fcc_qsro_256"] = {"cells": [256] * 3, "sites": Nq, "shells": 2, "composition": "Fe29Co29Ni28Al7Ti7",
                           "sweeps_per_launch": nswq, "launches_per_sweep": 256, "ms_per_sweep": msq / nswq,
                           "attempts_per_s": Nq * nswq / (msq * 1e-3),
                           "accept_rate": float(nq.item()) / (2 * Nq * nswq),
                           "paper_context_attempts_per_s": {"H100 SMC-X": 3.71e7, "H100 SMC-AI": 1.87e7}}
    eq = torch.zeros(1, dtype=torch.float64, device=dev)
    out["fcc_qsro_energy_256"] = {"ms": timed(lambda: smc.fcc_energy(latq, qm, occq, eq), reps=3)}
    del occq
    # dE/dtheta of the pair + MLP energy at 512^3 (one configuration)
    c5 = inputs.CONFIG5
    n5 = c5["cells"][0]
    lat5 = smc.Lattice(n5, n5, n5, S)
    occ5 = torch.empty(lat5.nsites, dtype=torch.int8, device=dev)
    smc.init_lattice(lat5, inputs.equiatomic_counts(lat5.nsites, S), c5["mc_seed"], occ5)
    m5 = smc.Model(smc.PAIR_F32_MLP_BF16, c5["nshells"], inputs.pair_f32_coeffs(c5["coeff_seed"], c5["nshells"], S),
                   mlp=inputs.mlp_weights(c5["mlp_seed"]))
    g5 = torch.zeros(smc.grad_size(lat5, m5), dtype=torch.float32, device=dev)
    gms5 = timed(lambda: smc.energy_grad(lat5, m5, occ5, g5), reps=2)
    tf5 = lat5.nsites * MLP_FLOP_PER_SITE_GRAD / (gms5 * 1e-3) / 1e12
    out["mlp_grad_512"] = {"cells": [n5] * 3, "ms_per_configuration": gms5, "params": int(g5.numel()),
                           "achieved_tflops": tf5, "frac_of_measured_bf16_sustained": tf5 / pk["bf16_tflops_sustained"],
                           "flop_per_site": MLP_FLOP_PER_SITE_GRAD}
    # Config 5 as a job: at 600 K, equilibration sweeps, then samples of (one
    # sweep, SRO of shells 1-3, dE/dtheta) and d<alpha>/dtheta from their
    # covariance.  The job has 20 + 200; a bounded part is timed here (2
    # equilibration sweeps, 4 samples) and the job's time extrapolated.
    kT5 = inputs.K_B_EV * c5["T"]
    n_eq, n_s = 2, 4
    A5 = torch.zeros((n_s, 3, S, S), dtype=torch.float64, device=dev)
    G5 = torch.zeros((n_s, g5.numel()), dtype=torch.float64, device=dev)
    cnt5 = torch.zeros((3, S, S), dtype=torch.int64, device=dev)
    al5 = torch.zeros((3, S, S), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(True) for _ in range(2 + 3 * n_s)]
    ev[0].record(stream)
    smc.sweep(lat5, m5, occ5, c5["mc_seed"], 0, n_eq, kT5)
    ev[1].record(stream)
    for i in range(n_s):
        ev[2 + 3 * i].record(stream)
        smc.sweep(lat5, m5, occ5, c5["mc_seed"], n_eq + i, 1, kT5)
        ev[3 + 3 * i].record(stream)
        smc.sro(lat5, 3, occ5, counts=cnt5, alpha=al5)
        smc.energy_grad(lat5, m5, occ5, g5)
        A5[i].copy_(al5)
        G5[i].copy_(g5)
        ev[4 + 3 * i].record(stream)
    torch.cuda.synchronize()
    smc.check()
    sw5 = float(np.mean([ev[2 + 3 * i].elapsed_time(ev[3 + 3 * i]) for i in range(n_s)]))
    ob5 = float(np.mean([ev[3 + 3 * i].elapsed_time(ev[4 + 3 * i]) for i in range(n_s)]))
    eq5 = ev[0].elapsed_time(ev[1]) / n_eq
    dadt = smc.observable_gradient(A5, G5, 1.0 / kT5)
    out["config5_512"] = {"cells": [n5] * 3, "T_K": c5["T"], "model": "FP32 2-shell pair + BF16 MLP",
                          "equilibration_sweeps_timed": n_eq, "samples_timed": n_s,
                          "ms_per_model_sweep": 0.5 * (eq5 + sw5),
                          "ms_per_configuration": ob5,
                          "ms_per_sample": sw5 + ob5,
                          "ratio_configuration_to_model_sweep": ob5 / sw5,
                          "ratio_configuration_to_plain_pair_sweep": ob5 / (ms / nsw),
                          "job_s_20_equilibration_200_samples": (20 * eq5 + 200 * (sw5 + ob5)) / 1e3,
                          "dalpha_dtheta_shape": list(dadt.shape),
                          "dalpha_dtheta_finite": bool(torch.isfinite(dadt).all()),
                          "note": "configuration = SRO (pair counts, alpha) + dE/dtheta (pair counts and the MLP "
                                  "adjoint); d<alpha>/dtheta = -beta cov(alpha, dE/dtheta) over the samples"}
    return out


if __name__ == "__main__":
    main()
