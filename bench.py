"""Benchmark of the fluctuating lattice Boltzmann step on GB300.

Default workload: D3Q19 force-based non-ideal fluid on a 256^3 periodic lattice
in FP32 deviation storage (A=-0.01, B=0.1, rho_c=1, kappa=0.02, kT=1e-6, all
relaxation rates 1, rho = 1 + U(-0.01, 0.01) from a seeded generator).  One
"step" is one full time step of the hot path: the density gather plus the fused
pull / MRT collide / force / Langevin-noise / store kernel.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun, one rank per GPU) every
rank advances its own independent replica (distinct Philox replica word):
weak scaling, no data-path collective.  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q19 fluctuating-LB MLUPS & % HBM roofline; batched/adjoint vs plain step"
UNIT = "MLUPS"
FE = dict(A=-0.01, B=0.1, rho_c=1.0, kappa=0.02)
WORKLOADS = {
    "nonideal256": dict(lattice=19, dims=(256, 256, 256), precision="fp32", fe=FE, kT=1e-6,
                        omega=(1.0, 1.0, 1.0), seed=3,
                        name="D3Q19 force-based non-ideal fluid, 256^3 periodic, FP32 deviations, "
                             "psi=A(rho-rho_c)^2/2+B(rho-rho_c)^4/4 (A=-0.01, B=0.1, rho_c=1), kappa=0.02, "
                             "F=-rho grad mu (19-point stencils), Guo forcing, kT=1e-6, omega_shear=1, "
                             "rho=1+U(-0.01,0.01)"),
    "nonideal128": dict(lattice=19, dims=(128, 128, 128), precision="fp32", fe=FE, kT=1e-6,
                        omega=(1.0, 1.0, 1.0), seed=3,
                        name="D3Q19 force-based non-ideal fluid, 128^3 periodic, FP32 deviations, "
                             "parameters of the 256^3 workload (profiling size)"),
    "nonideal256x256x128": dict(lattice=19, dims=(256, 256, 128), precision="fp32", fe=FE, kT=1e-6,
                                omega=(1.0, 1.0, 1.0), seed=3,
                                name="D3Q19 force-based non-ideal fluid, 256x256x128, FP32 (profiling size)"),
    "ideal256": dict(lattice=19, dims=(256, 256, 256), precision="fp32", fe=None, kT=1e-5,
                     omega=(1.2, 1.0, 1.0), seed=2,
                     name="D3Q19 ideal gas, 256^3 periodic, FP32 deviations, kT=1e-5, "
                          "omega=(1.2, 1.0, 1.0), shear wave + thermal start"),
    "capillary1024x400": dict(lattice=9, dims=(1024, 400, 1), precision="fp32",
                              fe=dict(A=-0.025, B=0.4, rho_c=0.75, kappa=0.08, total=True), kT=1e-7,
                              omega=(1.0, 1.0, 1.0), seed=11, stripe=200,
                              name="D2Q9 liquid stripe 1024x400 (thickness 200) of the Landau double well "
                                   "beta (rho-0.5)^2 (rho-1)^2, beta=0.1, kappa=0.08, as total bulk free energy "
                                   "(F = -rho grad mu + cs^2 grad rho), kT=1e-7, tau=1, FP32 deviations"),
    "swift1024x400": dict(lattice=9, dims=(1024, 400, 1), precision="fp32",
                          fe=dict(A=-0.025, B=0.4, rho_c=0.75, kappa=0.08, total=True, model=1), kT=1e-7,
                          omega=(1.0, 1.0, 1.0), seed=11, stripe=200,
                          name="D2Q9 liquid stripe 1024x400 (thickness 200) of the Landau double well "
                               "beta (rho-0.5)^2 (rho-1)^2, beta=0.1, kappa=0.08, modified-equilibrium model "
                               "(pressure in the equilibrium, e/eps noise coloured by FFT), kT=1e-7, tau=1, "
                               "FP32 deviations"),
    "nonideal256_bf16": dict(lattice=19, dims=(256, 256, 256), precision="bf16", fe=FE, kT=1e-6,
                             omega=(1.0, 1.0, 1.0), seed=3,
                             name="D3Q19 force-based non-ideal fluid, 256^3, BF16 deviations (FP32 arithmetic), "
                                  "parameters of the FP32 256^3 workload"),
    "ideal256_bf16": dict(lattice=19, dims=(256, 256, 256), precision="bf16", fe=None, kT=1e-5,
                          omega=(1.2, 1.0, 1.0), seed=2,
                          name="D3Q19 ideal gas, 256^3, BF16 deviations (FP32 arithmetic), kT=1e-5, "
                               "omega=(1.2, 1.0, 1.0), shear wave + thermal start"),
    "ideal128": dict(lattice=19, dims=(128, 128, 128), precision="fp32", fe=None, kT=1e-5,
                     omega=(1.2, 1.0, 1.0), seed=2,
                     name="D3Q19 ideal gas, 128^3 periodic, FP32 deviations, kT=1e-5, "
                          "omega=(1.2, 1.0, 1.0), shear wave + thermal start"),
}
# Algorithmic bytes per site and step of the path: every population is pulled
# (read) and stored once, and the non-ideal fluid also reads every population
# once more for the density gather, writes the density and reads it back (Q e +
# 2 e_rho).  The force-model steps (D3Q19 and D2Q9) do all of this in one launch
# and take the gather's re-reads and the density from L2 and shared memory, so
# their DRAM minimum is that of the ideal step (2 Q e); the modified-equilibrium
# step reads a density field and a noise field written before it.
ELEM = {"fp32": 4, "fp64": 8, "bf16": 2}
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def step_bytes(wl):
    """(algorithmic bytes per site of the step kernel, of the gather kernel,
    DRAM minimum per site of the step kernel)."""
    e = ELEM[wl["precision"]]
    Q = wl["lattice"]
    rb = 8 if wl["precision"] == "fp64" else 4
    if not wl["fe"]:
        return 2 * Q * e, 0, 2 * Q * e
    if wl["fe"].get("model", 0) == 1:  # + the density and the coloured e/eps noise field
        nf = 16 if wl["precision"] == "fp64" else 8
        return 2 * Q * e + rb + nf, Q * e + rb, 2 * Q * e + rb + nf
    return 3 * Q * e + 2 * rb, 0, 2 * Q * e


KERNEL_SOURCES = ("flb_device.cuh", "flb_kernels.cuh", "flb_prec.cuh")


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """Max of x over the ranks of the process group (x itself for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world: int, sites_per_rank: int, steps: int, seconds: float) -> float:
    """Site updates of all ranks per second, in millions (weak scaling: every
    rank advances its own lattice of sites_per_rank sites)."""
    return world * sites_per_rank * steps / seconds / 1e6


def replica_word(rank: int) -> int:
    """Fourth Philox counter word of the replica a rank advances (one per rank)."""
    return int(rank)


def sample_dims(wl, sites=262144):
    """Lattice of the CPU oracle's bounded sample, about `sites` sites (the
    modified-equilibrium oracle colours its noise with a direct DFT, so its
    sample is kept small)."""
    if wl["fe"] and wl["fe"].get("model", 0) == 1:
        sites = min(sites, 16384)
    if wl["lattice"] == 9:
        n = max(8, 2 * int(round(sites ** 0.5 / 2)))
        return (n, n, 1)
    n = max(8, 2 * int(round(sites ** (1 / 3) / 2)))
    return (n, n, n)


def initial_density(wl, dims):
    """Seeded initial density of a non-ideal workload (None for the ideal gas)."""
    from paper_1012_3632_gb300 import inputs

    if not wl["fe"]:
        return None
    if wl.get("stripe"):
        X, Y = dims[0], dims[1]
        th = wl["stripe"] * Y / wl["dims"][1]
        fe = wl["fe"]
        D = (-fe["A"] / fe["B"]) ** 0.5  # half the liquid-vapour gap of the double well
        rho_l, rho_v = fe["rho_c"] + D, fe["rho_c"] - D
        beta = fe["B"] / 4
        w = (8 * fe["kappa"] / beta) ** 0.5 / (rho_l - rho_v)
        return inputs.stripe_density(X, Y, rho_l, rho_v, w, 0.5 * (Y - th), 0.5 * (Y + th)).ravel()
    return inputs.uniform_density(dims, seed=wl["seed"])


def kernel_name(wl):
    """The step kernel the library launches for this workload."""
    packed = wl["precision"] in ("fp32", "bf16") and wl["dims"][0] % 2 == 0 and wl["lattice"] == 19
    if wl["fe"] and wl["fe"].get("model", 0) == 1:
        return "k_step_swift"
    if wl["fe"] and wl["lattice"] == 19:
        return "k_step_march2" if packed else "k_step_march"
    return "k_step2" if packed else "k_step"


def kernel_source_hash():
    """Hash of the sources the step kernels are compiled from (ncu counters taken
    on other sources are stale)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1012_3632_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(wl_key):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    or None when missing or taken on different kernel sources."""
    p = os.path.join(ROOT, "profiles", f"traffic_{wl_key}.json")
    try:
        j = json.load(open(p))
    except Exception:
        return None
    if j.get("kernel_source_hash") != kernel_source_hash():
        return None
    return j.get("dram_bytes_per_launch_full_size")


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples go to FLB_CLOCK_DIR (default: the system temp directory)
        d = os.environ.get("FLB_CLOCK_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def host_description():
    """Logical CPU count and CPU model of the host the oracle runs on."""
    import platform

    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


def cpu_baseline(wl, budget_s=12.0):
    """Time the FP64 oracle (single thread) on a periodic 64^3 (D3Q19) lattice with
    the workload's parameters; steps are added until about budget_s of CPU work."""
    import numpy as np

    import oracle
    from paper_1012_3632_gb300 import inputs

    dims = sample_dims(wl)
    om = wl["omega"]
    fe = wl["fe"] or {}
    p = oracle.Params(Q=wl["lattice"], dims=dims, omega_shear=om[0], omega_bulk=om[1], omega_ghost=om[2],
                      kT=wl["kT"], nonideal=bool(wl["fe"]), seed=wl["seed"], **fe)
    rho = initial_density(wl, dims)
    f = oracle.init(p, rho=rho, thermal=not wl["fe"])
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s or steps == 0:
        f = oracle.step(p, f, steps)
        steps += 1
    dt = time.perf_counter() - t0
    V = int(np.prod(dims))
    return {"value": V * steps / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{dims[0]}x{dims[1]}x{dims[2]} periodic lattice, same parameters, {steps} steps "
                      f"(about {budget_s:.0f} s of CPU work), FP64 C oracle, single thread",
            "host": host_description()}


def batched_vs_plain(n=64, steps=2000, every=20, seed=4):
    """The batched ensemble workload: 64 D3Q19 ideal-gas replicas, cubic sizes
    drawn from {32,48,64,96,128}, omega_shear ~ U(0.8,1.6), kT = 1e-5, FP32, one
    persistent launch per step replayed from a CUDA graph, 2000 steps with the
    ensemble observables accumulated in FP64 every 20 steps (every replica's
    mode variances and its density S(k) on the device).  Times the whole run,
    the steps alone, and the plain single-lattice step on the same replicas."""
    import numpy as np
    import torch

    from paper_1012_3632_gb300 import Batch, Context, inputs

    L = inputs.replica_sizes(n, seed=seed)
    om = inputs.replica_omegas(n, seed=seed)
    dims = [(int(l), int(l), int(l)) for l in L]
    sites = int(sum(l ** 3 for l in L))
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Batch(dims, om, [1e-5] * n, [1000 + r for r in range(n)], stream=stream.cuda_stream) as b:
        b.init(thermal=True)
        shapes = b.autotune()
        b.step(20)
        torch.cuda.synchronize()
        # the steps alone (graph replays)
        ev0.record(stream)
        b.step(200)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_batch = ev0.elapsed_time(ev1) / 200  # ms per ensemble step
        # the whole ensemble run: steps plus FP64 snapshot accumulation
        b.init(thermal=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps // every):
            b.step(every)
            var = b.mode_variance()
            for r in range(n):
                b.structure_factor(r, 0, accumulate=True, fetch=False)
        torch.cuda.synchronize()
        t_run = time.perf_counter() - t0
    kT = 1e-5
    N = np.array([1, 1 / 3, 1 / 3, 1 / 3, 2 / 3, 4 / 3, 4 / 9, 1 / 9, 1 / 9, 1 / 9, 2 / 27, 2 / 27, 2 / 27,
                  2 / 9, 2 / 9, 2 / 9, 2 / 9, 1 / 3, 1 / 9])
    T = (var / N / 3.0) / kT  # mode temperatures / kT, per replica
    # plain: one context per replica size, time per step times the count
    t_plain = 0.0
    for l in sorted(set(int(v) for v in L)):
        cnt = int((L == l).sum())
        with Context(19, (l, l, l), 1.2, kT=1e-5, seed=1, precision="fp32", stream=stream.cuda_stream) as c:
            c.init(thermal=True)
            c.step(10)
            torch.cuda.synchronize()
            ev0.record(stream)
            c.step(50)
            ev1.record(stream)
            torch.cuda.synchronize()
            t_plain += cnt * ev0.elapsed_time(ev1) / 50
    shape_of = {int(l): [int(v) for v in shapes[int(np.where(L == l)[0][0])]] for l in set(int(v) for v in L)}
    return {"workload": f"{n} D3Q19 ideal-gas replicas, cubic sizes from {{32,48,64,96,128}} (seed {seed}), "
                        "omega_shear U(0.8,1.6), kT=1e-5, FP32, graph-replayed persistent launch",
            "sites": sites, "batched_mlups": sites / (t_batch * 1e-3) / 1e6,
            "batched_gbs": 152 * sites / (t_batch * 1e-3) / 1e9,
            "plain_mlups": sites / (t_plain * 1e-3) / 1e6, "batched_over_plain": t_plain / t_batch,
            "ms_per_ensemble_step": t_batch, "tile_shape_per_size": shape_of,
            "ensemble_run": {"steps": steps, "snapshot_every": every, "seconds": t_run,
                             "mlups_with_snapshots": sites * steps / t_run / 1e6,
                             "what": "steps from a thermal start, every 20 steps flb_batch_mode_variance "
                                     "(all replicas, FP64) and flb_batch_structure_factor(mode 0, accumulate) "
                                     "for each replica on the device",
                             "mode_temperature_over_kT_ensemble_mean_range": [float(T[:, 4:].mean(0).min()),
                                                                               float(T[:, 4:].mean(0).max())]}}


def adjoint_vs_plain(dims=(64, 64, 64), nsteps=200, every=20, precision="fp32"):
    """Gradient workload: the 64^3 non-ideal fluid (parameters of the 256^3
    workload), 200 steps with checkpoints every 20, loss sum_k |rho_hat|^2
    exp(-k^2/0.5) at the last step.  Times the forward pass (steps +
    checkpoint copies), the backward pass (recomputation + adjoint steps) and
    the plain step on the same lattice."""
    import torch

    from paper_1012_3632_gb300 import Context, inputs
    from paper_1012_3632_gb300.adjoint import density_spectrum_loss, run

    V = dims[0] * dims[1] * dims[2]
    dt = torch.float32 if precision == "fp32" else torch.float64
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with Context(19, dims, 1.0, 1.0, 1.0, kT=1e-6, free_energy=FE, seed=5, precision=precision,
                 stream=stream.cuda_stream) as c:
        c.init(rho=inputs.uniform_density(dims, seed=5))
        c.step(20)
        torch.cuda.synchronize()
        ev[0].record(stream)
        c.step(nsteps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        t_plain = ev[0].elapsed_time(ev[1]) / nsteps
        g0 = torch.empty((19, V), dtype=dt, device="cuda")
        c.get_state_device(g0.data_ptr())
    cfg = dict(dims=dims, kT=1e-6, seed=5, precision=precision, nsteps=nsteps, every=every, nonideal=True, rho_c=1.0)
    # warm-up of the loss (cuFFT loads and plans on its first use) and of the
    # path, long enough for the step's column-length tuning
    density_spectrum_loss(g0, dims).item()
    warm = dict(cfg, nsteps=40, every=20)
    th0 = torch.tensor([1.0, 1.0, 1.0, 0.02, -0.01, 0.1], dtype=torch.float64, requires_grad=True)
    density_spectrum_loss(run(g0.clone().requires_grad_(True), th0, warm), dims).backward()
    theta = torch.tensor([1.0, 1.0, 1.0, 0.02, -0.01, 0.1], dtype=torch.float64, requires_grad=True)
    g = g0.clone().requires_grad_(True)
    torch.cuda.synchronize()
    ev[0].record(stream)
    loss = density_spectrum_loss(run(g, theta, cfg), dims)
    ev[1].record(stream)
    loss.backward()
    ev[2].record(stream)
    torch.cuda.synchronize()
    t_fwd = ev[0].elapsed_time(ev[1]) / nsteps
    t_bwd = ev[1].elapsed_time(ev[2]) / nsteps
    return {"workload": f"D3Q19 non-ideal {dims[0]}x{dims[1]}x{dims[2]} {precision.upper()}, {nsteps} steps, "
                        f"checkpoints every {every}, spectral density loss",
            "plain_ms_per_step": t_plain, "forward_ms_per_step": t_fwd, "backward_ms_per_step": t_bwd,
            "backward_over_plain": t_bwd / t_plain, "grad_theta": [float(v) for v in theta.grad]}


REF_BUDGET_S = 120.0  # wall-clock budget of the reference arm's warm-up + timed steps


def run_reference(args, wl, rank):
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1012_3632_gb300 import inputs

    om = wl["omega"]
    fe = wl["fe"] or {}

    def setup(dims):
        p = oracle.Params(Q=wl["lattice"], dims=dims, omega_shear=om[0], omega_bulk=om[1], omega_ghost=om[2],
                          kT=wl["kT"], nonideal=bool(wl["fe"]), seed=wl["seed"], **fe)
        return p, oracle.init(p, rho=initial_density(wl, dims), thermal=not wl["fe"])

    # size the per-step sample so that warm-up and timed steps take about
    # REF_BUDGET_S in total: time two steps of a small probe lattice first
    pdims = sample_dims(wl, 4096)
    p, f = setup(pdims)
    t0 = time.perf_counter()
    for t in range(2):
        f = oracle.step(p, f, t)
    per_site = (time.perf_counter() - t0) / (2 * np.prod(pdims))
    sites = REF_BUDGET_S / max(per_site, 1e-9) / (args.steps + args.warmup)
    dims = sample_dims(wl, int(min(262144, max(4096, sites))))
    p, f = setup(dims)
    for t in range(args.warmup):
        f = oracle.step(p, f, t)
    t0 = time.perf_counter()
    for t in range(args.steps):
        f = oracle.step(p, f, args.warmup + t)
    dt = time.perf_counter() - t0
    V = int(np.prod(dims))
    value = V * args.steps / dt / 1e6
    sample = f"{dims[0]}x{dims[1]}x{dims[2]} periodic lattice per step, same parameters, FP64 C oracle, 1 thread"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args, wl),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_description()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


L2_BYTES = 129e6  # GB300


def population_bytes(wl):
    return int(wl["dims"][0] * wl["dims"][1] * wl["dims"][2]) * wl["lattice"] * ELEM[wl["precision"]]


def flush_l2_between_steps(wl):
    """A step reads one population buffer; when that fits in L2 the timed steps
    are separated by an L2 flush instead."""
    return population_bytes(wl) <= L2_BYTES


def config_of(args, wl):
    V = int(wl["dims"][0] * wl["dims"][1] * wl["dims"][2])
    buf = population_bytes(wl)
    if flush_l2_between_steps(wl):
        l2 = (f"L2 flushed before every timed step (a {2 * L2_BYTES / 1e6:.0f} MB write outside the events); "
              f"population buffers of {buf / 1e9:.3g} GB each fit in L2")
    else:
        l2 = f"inputs larger than L2: two population buffers of {buf / 1e9:.3g} GB each, no flush"
    return {"workload": wl["name"], "lattice_sites": V, "dims": list(wl["dims"]), "replicas": args.gpus,
            "parallelism": f"replicas{args.gpus}", "l2": l2}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nonideal256", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-replica comparison")
    ap.add_argument("--batched-replicas", type=int, default=64, help="replicas of the batched ensemble")
    ap.add_argument("--batched-steps", type=int, default=2000, help="ensemble steps with snapshots")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    wl = WORKLOADS[args.workload]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, wl, rank)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1012_3632_gb300 import Context, RHO, inputs
    from paper_1012_3632_gb300 import build as B

    B.build()
    stream = torch.cuda.current_stream()
    om = wl["omega"]
    dims = wl["dims"]
    V = dims[0] * dims[1] * dims[2]
    ctx = Context(wl["lattice"], dims, om[0], om[1], om[2], kT=wl["kT"], free_energy=wl["fe"], seed=wl["seed"],
                  precision=wl["precision"], replica=replica_word(rank), stream=stream.cuda_stream, device=local)
    rho = initial_density(wl, dims)
    u = None if wl["fe"] else inputs.shear_wave(dims, amp=1e-3)
    ctx.init(rho=rho, u=u, thermal=not wl["fe"])

    # ---- device-resident timing ------------------------------------------
    # setup: the z-marching step times its candidate column lengths on its
    # first launches; finish that before the warm-up steps so that the timed
    # steps all run with the chosen length
    n_tune = 0
    while ctx.z_chunk()[1] and n_tune < 256:
        ctx.step(1)
        n_tune += 1
    ctx.step(args.warmup)
    ctx.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush = flush_l2_between_steps(wl)
    if flush:
        scratch = torch.empty(int(2 * L2_BYTES) // 4, dtype=torch.float32, device=f"cuda:{local}")
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    # the library brackets every step-kernel launch with CUDA events on its
    # stream (flb_kernel_timing) inside the timed region, so the kernel's own
    # time is part of, and never exceeds, the step time
    ctx.kernel_timing(True)
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        barrier()
        torch.cuda.synchronize()
        if flush:
            for k, (e0, e1) in enumerate(evs):
                scratch.fill_(float(k))
                e0.record(stream)
                ctx.step(1)
                e1.record(stream)
        else:
            ev0.record(stream)
            ctx.step(args.steps)
            ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) if flush else ev0.elapsed_time(ev1)
    kms, kn = ctx.kernel_times()
    ctx.kernel_timing(False)
    n_kt = args.steps
    z_planes, z_tuning = ctx.z_chunk()
    ms_max = max_over_ranks(ms, world)
    value = whole_job_mlups(world, V, args.steps, ms_max * 1e-3)

    # ---- end to end through the C ABI with host buffers ---------------------
    # the initial density field (pinned host -> device) in; every step
    # flb_step_sums_async: the step and the copy of its result, the FP64 mass
    # and momentum sums of the state it starts from (32 bytes device ->
    # page-locked host), without a wait per step; the density field out (that
    # read waits for the stream, so every step's sums are then in host memory).
    host_in = torch.empty(V, dtype=torch.float64, pin_memory=True).numpy()
    host_out = torch.empty(V, dtype=torch.float64, pin_memory=True).numpy()
    host_in[:] = rho if rho is not None else 1.0
    sums = torch.empty((args.steps, 4), dtype=torch.float64, pin_memory=True).numpy()

    def end_to_end(sync_each_step):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if wl["fe"]:
            ctx.init(rho=host_in)
        else:
            ctx.init(rho=host_in, u=u, thermal=True)
        for t in range(args.steps):
            if sync_each_step:
                ctx.step_sums(1, out=sums[t:t + 1])
            else:
                ctx.step_sums_async(1, sums[t])
        ctx.moments(RHO, out=host_out)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    t_e2e = end_to_end(False)
    e2e_value = whole_job_mlups(world, V, args.steps, max_over_ranks(t_e2e, world))
    drift = float(abs(sums[-1, 0] - sums[0, 0]) / abs(sums[0, 0]))
    t_sync = end_to_end(True)
    bytes_u = 0 if wl["fe"] else 3 * V * 8
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": (V * 8 + bytes_u) / args.steps,
           "d2h_bytes_per_step": 32 + V * 8 / args.steps,
           "what": "flb_init from a pinned host density field; per step flb_step_sums_async (the step, and the "
                   "copy of the FP64 mass and momentum of the state it starts from into page-locked host memory, "
                   "without a per-step wait); flb_moments(RHO) to pinned host at the end, which waits for all of it",
           "mass_drift": drift,
           "sync_each_step": {"value": whole_job_mlups(world, V, args.steps, max_over_ranks(t_sync, world)),
                              "what": "the same with flb_step_sums, which waits for each step's sums",
                              "host_round_trip_ms_per_step": (t_sync - t_e2e) * 1e3 / args.steps}}

    ctx.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    fused_b, gather_b, fused_min = step_bytes(wl)
    peak, peak_kind = measured_peak()
    n_fused = int(kn[1])
    t_fused = kms[1] / max(n_fused, 1) * 1e-3
    achieved = fused_b * V / t_fused / 1e9
    traffic = ncu_traffic(args.workload)
    # kernels per step: the timed kinds (gather, step, checks), plus, for the
    # modified-equilibrium noise, its white draw, colouring and two 2-D FFTs
    per_step = (kn[0] + kn[1] + kn[2]) / max(n_kt, 1)
    if wl["fe"] and wl["fe"].get("model", 0) == 1 and wl["kT"] > 0:
        per_step += 6
    n_launch = int(round(per_step * args.steps))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "bf16"}[wl["precision"]],
        "data": "synthetic", "config": config_of(args, wl),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": f"{peak_kind} copy bandwidth",
                     "kernel": kernel_name(wl),
                     "what": "fused pull + moment-space MRT collide + Guo force + Philox/Box-Muller noise + store",
                     "bytes_per_site": fused_b, "sites_per_launch": V,
                     "avg_launch_ms": t_fused * 1e3,
                     "dram_min_bytes_per_site": fused_min,
                     "frac_of_dram_min": fused_min * V / t_fused / 1e9 / peak,
                     "achieved_dram_gbs": traffic / t_fused / 1e9 if traffic else None,
                     "frac_dram": traffic / t_fused / 1e9 / peak if traffic else None,
                     "dram_bytes_per_site": traffic / V if traffic else None},
        "kernels": {"density_gather": {"launches": int(kn[0]), "avg_ms": kms[0] / max(kn[0], 1),
                                       "bytes_per_site": gather_b,
                                       "achieved_gbs": gather_b * V / (kms[0] / max(kn[0], 1) * 1e-3) / 1e9
                                       if kn[0] else None},
                    "fused_step": {"launches": n_fused, "avg_ms": kms[1] / max(n_fused, 1)},
                    "timed_with_events_over_steps": n_kt,
                    "z_planes_per_block": z_planes, "z_chunk_tuning_steps_before_warmup": n_tune,
                    "z_chunk_tuned_before_timing": not z_tuning},
        "whole_step_gbs": (fused_b + gather_b) * V / (ms_max / args.steps * 1e-3) / 1e9,
        "clocks": clk.summary(), "e2e": e2e, "gpu_launches": n_launch,
    }
    if not args.no_batched:
        line["batched"] = batched_vs_plain(n=args.batched_replicas, steps=args.batched_steps)
        line["adjoint"] = adjoint_vs_plain()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
