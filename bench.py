"""Throughput of the fused DDF stream-and-collide update on the stratified
Taylor-Green vortex, in MLUPS (million lattice-node updates per second) and as
a fraction of the measured HBM roofline.

Workload: 256^3 periodic box, D3Q27 momentum x D3Q19 scalar stencils,
Shan-Chen velocity-shift forcing, Re 800, Fr 0.1, Pr (= Sc) 1, U0 = 0.04,
diagnostics (E_k, E_p, eps_k, eps_p) every 100 steps. One bench step is one
diagnostics interval: 100 lattice updates plus one diagnostics evaluation,
whose per-node part is fused into the first update (lbm_step_diagnostics).
`value` is FP32-storage MLUPS over the timed steps; FP16/BF16 deviation
storage (FP32 arithmetic) is timed the same way and reported beside it with
the library's 16-bit storage rule applied to whole diagnostics series. The
64-instance sweep of the batched drivers follows.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       python bench.py --validation all      (the paper's own runs at 256^3)
Under torchrun (N > 1) each rank advances its own replica of the headline
lattice (the z-slab split with halo exchange exists, halo.py, but the
headline number stays a per-GPU replica); `value` sums the ranks' node
updates over the max per-rank time. The batch sweep is split over the ranks
(lbm_batch_partition), the whole sweep's updates over the slowest rank.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 256
PAIR = "27x19"
FORCING = "sc"
RE, FR, PR, U0 = 800.0, 0.1, 1.0, 0.04
DIAG_EVERY = 100
METRIC = "DDF MLUPS (FP32 storage) & % of HBM roofline; FP16-storage vs FP32 at <=1% KE/PE/eps error"
WORKLOAD = "stratified TGV 256^3, D3Q27xD3Q19, velocity-shift (Shan-Chen) forcing, Re 800, Fr 0.1, Pr 1, U0 0.04"


# DRAM bytes per step-kernel launch on the 256^3 bench lattice
# (dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture, mean of
# an even and an odd launch), with the fingerprint of the kernel sources the
# capture ran; reported as null once the sources differ from it.
NCU_TRAFFIC = {"fingerprint": "18dee20ce526b74c", "fp32": 6116793728, "fp16": 3027879552, "bf16": 3028134272}


def source_fingerprint() -> str:
    """Hash of the sources that define the bench's step kernels: the device
    headers and the D3Q27xD3Q19 instantiations (the host-side launch code, the
    staged kernel's header and the other stencil pairs' instantiations are not
    part of it)."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2605_14505_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        # the staged kernel's header does not enter the direct step kernels' code
        if (name.endswith(".cuh") and name != "lbm_stage.cuh") or name.startswith("inst_q27q19_") \
                or name == "lbm_dispatch.h":
            with open(os.path.join(csrc, name), "rb") as fh:
                h.update(name.encode())
                h.update(fh.read())
    return h.hexdigest()[:16]


# DRAM bytes per step of the 64-instance sweep, by driver (ncu, on the step
# kernels of the fingerprint above): the per-instance driver over 128
# graph-replayed steps as one profiler range (--replay-mode app-range, all
# streams together: 739.9 GB in 128 steps, the instances' own L2 reuse
# included); the persistent driver from one launch of 4 steps (5.97 GB per
# step, the algorithmic 5.95 GB).
NCU_BATCH_DRAM = {"fingerprint": "18dee20ce526b74c", "instances": 5780572946, "persistent": 5971162432}


def ncu_traffic(storage: str):
    if NCU_TRAFFIC["fingerprint"] != source_fingerprint():
        return None
    return NCU_TRAFFIC.get(storage)


def bytes_per_node(storage: str) -> int:
    # every population read once and written once per update
    return (27 + 19) * 2 * (4 if storage == "fp32" else 2)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    """Rank layout from the torchrun environment; one process group per job
    (NCCL with GPUs, gloo without), used only for barriers and the max-time
    reduction: the replicas exchange no lattice data."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(units_per_rank: float, world: int, max_secs: float) -> float:
    """Whole-job throughput: every rank's lattice-node updates over the slowest
    rank's time (weak scaling: each replica does the same work)."""
    return units_per_rank * world / max_secs / 1e6


def run_gpu_arm(args):
    import numpy as np
    import torch

    import stgv_inputs as inputs
    from paper_2605_14505_gb300 import lbm

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    n3 = N ** 3
    peak, peak_kind = measured_peaks()

    def make(storage):
        p = lbm.lbm_params_from_physics(N, N, N, PAIR, FORCING, RE, FR, PR, U0)
        sim = lbm.Simulation(p, storage=storage)
        sim.init_tgv(seed=1, noise_amp=1e-3)
        return sim

    def timed(sim, steps, warmup):
        """Seconds for `steps` bench steps, mean step-kernel launch ms, last diag.

        A bench step is one diagnosing step (lbm_step_diagnostics: the
        diagnostics of the state, reduced by the step kernel that loads it,
        plus the gradient and final passes) and DIAG_EVERY - 1 plain steps,
        whose launches are bracketed by CUDA events on the library's stream."""
        stream = torch.cuda.ExternalStream(sim.stream.cuda_stream)
        for _ in range(warmup):
            sim.step_diagnostics(1)
            sim.step(DIAG_EVERY - 1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        sim.synchronize()
        torch.cuda.synchronize()
        barrier(world)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        d = None
        for k in range(steps):
            d = sim.step_diagnostics(1)
            ev[k][0].record(stream)
            sim.step(DIAG_EVERY - 1)
            ev[k][1].record(stream)
        t1.record(stream)
        sim.synchronize()
        torch.cuda.synchronize()
        barrier(world)
        total_ms = t0.elapsed_time(t1)
        step_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / (steps * (DIAG_EVERY - 1))
        diag_ms = total_ms / steps - (DIAG_EVERY - 1) * step_ms   # diagnosing step + passes 2, 3
        return total_ms / 1e3, step_ms, diag_ms, d

    clocks = ClockSampler(local)
    sim = make("fp32")
    bx, by = lbm.lbm_get_block(sim.h)
    clocks.start()
    secs, step_ms, diag_ms, d32 = timed(sim, args.steps, args.warmup)
    clk = clocks.stop()
    secs = max_over_ranks(world, secs)
    value = aggregate_mlups(float(n3) * DIAG_EVERY * args.steps, world, secs)
    achieved = bytes_per_node("fp32") * n3 / (step_ms * 1e-3) / 1e9
    sim.close()

    variants = {}
    for storage in ("fp16", "bf16"):
        s = make(storage)
        vsecs, vstep_ms, _, dv = timed(s, args.steps, args.warmup)
        vsecs = max_over_ranks(world, vsecs)
        vmlups = aggregate_mlups(float(n3) * DIAG_EVERY * args.steps, world, vsecs)
        vach = bytes_per_node(storage) * n3 / (vstep_ms * 1e-3) / 1e9
        err = {k: abs(dv[k] - d32[k]) / abs(d32[k]) for k in ("Ek", "Ep", "eps_k", "eps_p")}
        variants[storage] = {
            "mlups": round(vmlups, 1), "speedup_vs_fp32": round(vmlups / value, 3),
            "step_kernel_ms": round(vstep_ms, 4),
            "roofline": {"bound": "hbm", "achieved": round(vach, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(vach / peak, 4), "traffic": ncu_traffic(storage),
                         "algorithmic_bytes_per_launch": bytes_per_node(storage) * n3},
            "rel_dev_vs_fp32_gpu_at_last_timed_step": {k: float(f"{v:.3e}") for k, v in err.items()},
            "bytes_per_node": bytes_per_node(storage),
        }
        s.close()

    # the 16-bit storage rule (lbm_storage_rule, <= 1 % on E_k, E_p, eps_k,
    # eps_p and the two eps peaks, else FP32) on whole series: against the
    # stored FP64 oracle series of the 64^3 runs, and on this workload's full
    # 20000 steps against its FP32 run (no oracle at 256^3)
    if not args.no_series:
        precision = storage_rule_series(args)
        for storage in ("fp16", "bf16"):
            variants[storage]["storage_rule"] = precision[storage]

    # end to end through the C ABI with host buffers: every bench step sets the
    # lattice from FP64 fields in pinned host memory, advances 100 steps and
    # reads a diagnostics record back: that of the state after 99 steps,
    # reduced by the 100th step, which loads it anyway (lbm_step_diagnostics),
    # so the GPU work is the timed device loop's plus the initialisation.
    # Pipelined as a user streaming states would run it: the host-to-device
    # copy of the next step's fields (lbm_prefetch_fields, a side stream)
    # overlaps the current steps.
    rho, u, rp = inputs.tgv_fields(N, U0, seed=1, noise_amp=1e-3)
    hr = torch.from_numpy(rho).pin_memory()
    hu = torch.from_numpy(np.ascontiguousarray(u)).pin_memory()
    hp = torch.from_numpy(rp).pin_memory()
    p = lbm.lbm_params_from_physics(N, N, N, PAIR, FORCING, RE, FR, PR, U0)
    h = lbm.lbm_create_params(p)

    def e2e_step():
        lbm.lbm_init_prefetched(h)
        lbm.lbm_prefetch_fields(h, hr, hu, hp)   # the next bench step's inputs
        lbm.lbm_step(h, DIAG_EVERY - 1)
        return lbm.lbm_step_diagnostics(h, 1)

    lbm.lbm_prefetch_fields(h, hr, hu, hp)
    for _ in range(args.warmup):
        e2e_step()
    lbm.lbm_synchronize(h)
    barrier(world)
    t = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    lbm.lbm_synchronize(h)
    barrier(world)
    e2e_secs = max_over_ranks(world, time.perf_counter() - t)
    lbm.lbm_destroy(h)
    e2e = {"value": round(aggregate_mlups(float(n3) * DIAG_EVERY * args.steps, world, e2e_secs), 1),
           "unit": "MLUPS", "h2d_bytes_per_step": 5 * n3 * 8, "d2h_bytes_per_step": 11 * 8}

    batch = run_batch_sweep(args, peak, world, rank) if not args.no_batch else None

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (Eq. 20 Taylor-Green field + 1e-3 U0 SplitMix64 noise)",
        "config": {"workload": WORKLOAD, "lattice": [N, N, N], "pair": "D3Q27xD3Q19", "forcing": "shan_chen",
                   "storage": "fp32", "updates_per_step": DIAG_EVERY, "diagnostics_per_step": 1,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (3.09 GB store vs 129 MB L2)", "block": [bx, by]},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": ncu_traffic("fp32"),
                     "algorithmic_bytes_per_launch": bytes_per_node("fp32") * n3,
                     "kernel": "k_step<27x19, SC, f32> (even/odd AA)", "peak_kind": peak_kind,
                     "bytes_per_node": bytes_per_node("fp32"), "step_kernel_ms": round(step_ms, 4),
                     "diagnosing_step_ms": round(diag_ms, 4)},
        "storage_variants": variants,
        "batch": batch,
        "e2e": e2e,
        "gpu_launches": args.steps * (DIAG_EVERY + 3),
        "clocks": clk,
    }
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_steps)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


SERIES_STEPS, SERIES_EVERY = 20000, 100


def _series(n, pair, forcing, Re, Fr, Sc, U0_, steps, every, seed, amp, storage, host_fields):
    """Diagnostics every `every` steps (lbm_step_diagnostics) from step 0 to `steps`."""
    import stgv_inputs as inputs
    from paper_2605_14505_gb300 import lbm

    p = lbm.lbm_params_from_physics(n, n, n, pair, forcing, Re, Fr, Sc, U0_)
    sim = lbm.Simulation(p, storage=storage)
    if host_fields:
        sim.init_fields(*inputs.tgv_fields(n, U0_, seed=seed, noise_amp=amp))
    else:
        sim.init_tgv(seed=seed, noise_amp=amp)
    out = [sim.step_diagnostics(every, allow_nonfinite=True) for _ in range(steps // every)]
    out.append(sim.diagnostics(allow_nonfinite=True))
    sim.close()
    return out


def storage_rule_series(args) -> dict:
    """FP16 and BF16 deviation storage judged by the library's storage rule:
      - against the FP64 oracle: the stored oracle series of two 64^3 runs
        (written by tests/golden/make_oracle_series.py; no oracle code runs
        here): Re 200 / Fr 0.1 (laminar) and the paper's Re0 1600 / Fr0 1
        (turbulent breakdown, t ~ 30);
      - on the 256^3 workload's full 20000 steps (diagnostics every 100)
        against the FP32-storage run on this GPU."""
    import importlib.util

    from paper_2605_14505_gb300 import lbm

    spec = importlib.util.spec_from_file_location(
        "make_oracle_series", os.path.join(ROOT, "tests", "golden", "make_oracle_series.py"))
    G = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(G)
    keys = ("dev_Ek", "dev_Ep", "dev_eps_k", "dev_eps_p", "dev_peak1", "dev_peak2")

    def brief(rep):
        d = {k: float(f"{rep[k]:.3e}") for k in keys}
        d.update(selected=rep["selected"], step_peak1=rep["step_peak1"], step_peak2=rep["step_peak2"])
        return d

    res = {"fp16": {}, "bf16": {}}
    for name in ("stgv64_re200_fr01_sc", "stgv64_paper_re1600_fr1_sc"):
        n, (qf, qg), forcing, Re, Fr, Sc, U0_, steps, every, seed, amp = G.SERIES[name]
        ref = G.read(name)
        for storage in res:
            got = _series(n, f"{qf}x{qg}", forcing, Re, Fr, Sc, U0_, steps, every, seed, amp, storage, True)
            for d, r in zip(got, ref):
                assert d["step"] == r["step"]
            res[storage]["vs_fp64_oracle_" + name] = brief(lbm.lbm_storage_rule(ref, got, storage, 0.01))
    if args.series_steps > 0:
        ref = _series(N, PAIR, FORCING, RE, FR, PR, U0, args.series_steps, SERIES_EVERY, 1, 1e-3, "fp32", False)
        for storage in res:
            got = _series(N, PAIR, FORCING, RE, FR, PR, U0, args.series_steps, SERIES_EVERY, 1, 1e-3, storage, False)
            rep = brief(lbm.lbm_storage_rule(ref, got, storage, 0.01))
            rep["steps"] = args.series_steps
            res[storage]["vs_fp32_gpu_256cubed_workload"] = rep
    for storage in res:
        res[storage]["verdict"] = "kept" if all(v["selected"] == storage for v in res[storage].values()) \
            else "fp32 fallback"
    return res


SWEEP_STEPS = 2000


def sweep_specs():
    """64 independent lattices: sizes {32, 48, 64, 96}^3 x Fr {1, 0.5, 0.2, 0.1}
    x forcing {Guo, Shan-Chen} x pair {D3Q19xD3Q7, D3Q27xD3Q19}, Re 200, Pr 1, U0 0.04."""
    return [(n, pair, forcing, 200.0, fr) for n in (32, 48, 64, 96) for fr in (1.0, 0.5, 0.2, 0.1)
            for forcing in ("guo", "sc") for pair in ("19x7", "27x19")]


def run_batch_sweep(args, peak, world=1, rank=0):
    """The 64 instances advanced together for 2000 steps, driver and launch
    shapes picked by the library's autotuner. Aggregate MLUPS and the HBM
    roofline fraction of the whole batch. Under torchrun the instances are
    split over the ranks by lbm_batch_partition (bytes per step, longest
    first): each rank advances only its own, with no lattice data exchanged,
    and the job's time is the slowest rank's (the sweep's total work is fixed:
    strong scaling)."""
    import numpy as np
    import torch

    from paper_2605_14505_gb300 import lbm

    specs = sweep_specs()
    params_all = [lbm.lbm_params_from_physics(n, n, n, pair, f, Re, Fr, 1.0, U0) for n, pair, f, Re, Fr in specs]
    owner, imbalance = lbm.lbm_batch_partition(params_all, world)
    mine = [i for i in range(len(specs)) if owner[i] == rank]
    params = [params_all[i] for i in mine]
    b = lbm.lbm_batch_create(params)
    lbm.lbm_batch_init_tgv(b, seed=1, noise_amp=1e-3)
    tuned_ms = lbm.lbm_batch_autotune(b, 3)
    cfg = lbm.lbm_batch_get_config(b)
    flow_nodes = lbm.lbm_batch_get_flow_nodes(b)
    lbm.lbm_batch_step(b, 100)
    lbm.lbm_batch_synchronize(b)
    barrier(world)
    t = time.perf_counter()
    steps = args.sweep_steps
    lbm.lbm_batch_step(b, steps)
    lbm.lbm_batch_synchronize(b)
    secs = max_over_ranks(world, time.perf_counter() - t)
    nodes = sum(n ** 3 for n, *_ in specs)
    nbytes = sum(n ** 3 * (bytes_per_node("fp32") if pair == "27x19" else (19 + 7) * 2 * 4)
                 for n, pair, *_ in specs)
    diags = lbm.lbm_batch_diagnostics(b)
    lbm.lbm_batch_destroy(b)
    torch.cuda.synchronize()
    finite = all(np.isfinite(d["Ek"]) for d in diags)
    if world > 1:
        finite = max_over_ranks(world, 0.0 if finite else 1.0) == 0.0
    achieved = nbytes * steps / secs / 1e9
    drivers = {0: "persistent", 1: "per_step", 2: "instances"}
    driver = drivers[cfg["mode"]]
    dram = NCU_BATCH_DRAM.get(driver) if NCU_BATCH_DRAM["fingerprint"] == source_fingerprint() else None
    roof = {"bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
            "traffic": dram, "algorithmic_bytes_per_step": nbytes,
            "achieved_algorithmic": round(achieved, 1), "frac_algorithmic": round(achieved / peak / world, 4),
            "counts": "achieved / frac: DRAM bytes per step (ncu, traffic) over the measured step time; "
                      "*_algorithmic: every population read and written once per step"}
    if dram is not None:
        # the whole sweep's DRAM bytes per step (split over the ranks when there are several)
        roof["achieved"] = round(dram * steps / secs / 1e9, 1)
        roof["frac"] = round(dram * steps / secs / 1e9 / (peak * world), 4)
    return {"instances": len(specs), "nodes": nodes, "steps": steps,
            "mlups": round(nodes * steps / secs / 1e6, 1), "ms_per_step": round(secs * 1e3 / steps, 4),
            "roofline": roof,
            "driver": driver,
            "tile": [cfg["bx"], cfg["by"]] if cfg["mode"] == 1 else None,
            "flow_nodes": flow_nodes if cfg["mode"] == 0 else None,
            "autotune_ms_per_step": round(tuned_ms, 4),
            "ranks": world, "instances_this_rank": len(mine), "partition_imbalance": round(imbalance, 4),
            "scaling": "strong (the 64 instances split over the ranks)" if world > 1 else None,
            "all_finite": finite, "timing": f"host wall clock around {steps} steps, max over ranks"}


def cpu_baseline(steps: int = 2) -> dict:
    """The FP64 oracle as it stands on this host's cores: `steps` time steps of
    the same 256^3 lattice (initialisation not timed)."""
    import stgv_inputs as inputs
    from oracle import oracle

    p = oracle.params_from_physics(N, 27, 19, FORCING, RE, FR, PR, U0)
    sim = oracle.OracleSim(p)
    sim.init_fields(*inputs.tgv_fields(N, U0, seed=1, noise_amp=1e-3))
    t = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t
    sim.close()
    return {"value": round(N ** 3 * steps / dt / 1e6, 3), "unit": "MLUPS", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{steps} time steps of the full {N}^3 lattice, FP64, "
                                        "two-lattice pull streaming (init not timed)"}


def run_reference_arm(args):
    """The FP64 CPU oracle timed on the host cores on the same workload; each
    bench step is one time step of the 256^3 lattice (a bounded sample of the
    100-update diagnostics interval)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import stgv_inputs as inputs
    from oracle import oracle

    p = oracle.params_from_physics(N, 27, 19, FORCING, RE, FR, PR, U0)
    sim = oracle.OracleSim(p)
    sim.init_fields(*inputs.tgv_fields(N, U0, seed=1, noise_amp=1e-3))
    sim.step(args.warmup)
    t = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t
    sim.close()
    value = N ** 3 * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Eq. 20 Taylor-Green field + 1e-3 U0 SplitMix64 noise)",
        "config": {"workload": WORKLOAD, "lattice": [N, N, N], "pair": "D3Q27xD3Q19", "forcing": "shan_chen",
                   "storage": "fp64", "updates_per_step": 1, "parallelism": "host cores"},
        "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"{args.steps} time steps of the full {N}^3 lattice per run, FP64"},
        "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_ncu_case(args):
    """A small case for ncu captures (no timing output): an n^3 lattice of the
    bench's physics with the given storage or stencil pair, initialised and
    advanced `ncu_steps` single-kernel steps (graph replay off, so every step
    is its own launch), then one diagnostics evaluation."""
    import torch

    from paper_2605_14505_gb300 import lbm

    if args.ncu_case == "batch-inst":
        # the 64-instance sweep under the per-instance driver (each instance's
        # own step kernel and default launch shapes, no autotuning): init,
        # then ncu_steps steps, for a bounded launch list with DRAM bytes
        specs = sweep_specs()
        params = [lbm.lbm_params_from_physics(n, n, n, pair, f, Re, Fr, 1.0, U0) for n, pair, f, Re, Fr in specs]
        b = lbm.lbm_batch_create(params)
        lbm.lbm_batch_set_mode(b, "instances")
        lbm.lbm_batch_init_tgv(b, seed=1, noise_amp=1e-3)
        if args.ncu_range:
            # warm the caches and graphs, then bracket the measured steps with
            # cudaProfilerStart/Stop (an ncu range, all streams together)
            lbm.lbm_batch_step(b, args.ncu_steps)
            lbm.lbm_batch_synchronize(b)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
        lbm.lbm_batch_step(b, args.ncu_steps)
        lbm.lbm_batch_synchronize(b)
        if args.ncu_range:
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        lbm.lbm_batch_destroy(b)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": args.ncu_case, "steps": args.ncu_steps, "sources": source_fingerprint()}))
        return
    if args.ncu_case in ("batch", "batch-step"):
        # the 64-instance sweep: persistent driver, `ncu_steps` steps per launch;
        # or the per-step driver (one launch per variant and step, below the
        # graph length, so every launch is a plain one) with its 32 x 2 tiles
        specs = sweep_specs()
        params = [lbm.lbm_params_from_physics(n, n, n, pair, f, Re, Fr, 1.0, U0) for n, pair, f, Re, Fr in specs]
        b = lbm.lbm_batch_create(params)
        if args.ncu_case == "batch":
            lbm.lbm_batch_set_mode(b, "persistent", args.ncu_steps)
            lbm.lbm_batch_set_block(b, 32, 8)
        else:
            lbm.lbm_batch_set_mode(b, "per_step")
            lbm.lbm_batch_set_block(b, 32, 2)
        lbm.lbm_batch_init_tgv(b, seed=1, noise_amp=1e-3)
        lbm.lbm_batch_step(b, 3 * args.ncu_steps)
        lbm.lbm_batch_synchronize(b)
        lbm.lbm_batch_destroy(b)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": args.ncu_case, "steps": 3 * args.ncu_steps, "sources": source_fingerprint()}))
        return
    storage, pair = args.ncu_case, PAIR
    if args.ncu_case.startswith("19x7"):
        storage, pair = ("fp16" if args.ncu_case.endswith("fp16") else "fp32"), "19x7"
    p = lbm.lbm_params_from_physics(args.ncu_n, args.ncu_n, args.ncu_n, pair, FORCING, RE, FR, PR, U0)
    sim = lbm.Simulation(p, storage=storage)
    lbm.lbm_set_graphs(sim.h, False)
    lbm.lbm_set_pairing(sim.h, args.ncu_pairing)
    lbm.lbm_set_tile_staging(sim.h, args.ncu_staging)
    sim.init_tgv(seed=1, noise_amp=1e-3)
    sim.step(args.ncu_steps)
    d = sim.diagnostics()
    sim.close()
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": args.ncu_case, "n": args.ncu_n, "steps": args.ncu_steps, "Ek": d["Ek"],
                      "sources": source_fingerprint()}))


PAPER = {"n": 256, "pair": "27x19", "forcing": "sc", "Re": 1600.0, "Sc": 0.7, "U0": 0.0577}
FROUDE = (1.0, 0.1, 0.3, 0.5, 0.9, 1.5, 2.5)
X1_RE = (100.0, 200.0, 400.0, 800.0, 1600.0, 3000.0)
X1_U0 = 0.05 / 3 ** 0.5   # Ma 0.05 (Section 3.1)


def paper_series(n, pair, forcing, Re, Fr, Sc, U0, t_end, storage="fp32", seed=1, noise_amp=0.0,
                 spectrum_at=None, every_tc=0.1, pressure=False):
    """Diagnostics every ~every_tc convective times to t_end (lbm_step_diagnostics:
    reduced inside the step kernel), and optionally the kinetic-energy spectrum of
    the first sample at t >= spectrum_at (fields written to device memory, cuFFT).
    pressure: start from rho = 1 + p / cs^2 with the Taylor-Green pressure
    instead of rho = 1 (fewer sound waves at the start)."""
    import stgv_inputs as inputs
    from paper_2605_14505_gb300 import lbm, post

    p = lbm.lbm_params_from_physics(n, n, n, pair, forcing, Re, Fr, Sc, U0)
    sim = lbm.Simulation(p, storage=storage)
    if pressure:
        _, u, rp = inputs.tgv_fields(n, U0, seed=seed, noise_amp=noise_amp)
        sim.init_fields(post.tgv_pressure_density(n, U0), u, rp)
    else:
        sim.init_tgv(seed=seed, noise_amp=noise_amp)
    steps_tc = p.L / U0
    every = max(1, round(every_tc * steps_tc))
    total = round(t_end * steps_tc)
    series, spec = [], None
    t0 = time.perf_counter()
    while sim.step_count <= total:
        if spectrum_at is not None and spec is None and sim.step_count * U0 / p.L >= spectrum_at:
            _, u, _ = sim.fields_device()
            k, E = post.energy_spectrum_device(u, n)
            spec = {"t": sim.step_count * U0 / p.L, "k": k.tolist(), "E_phys": (E / U0 ** 2).tolist()}
        series.append(sim.step_diagnostics(every, allow_nonfinite=True))
        if not all(map(lambda v: v == v, (series[-1]["Ek"], series[-1]["eps_k"]))):
            break
    sim.synchronize()
    secs = time.perf_counter() - t0
    sim.close()
    return series, spec, secs


def run_validation(args):
    """The paper's own runs at 256^3 on one GPU (context, not gates: the paper's
    DNS references are not available):
      - X1 (Section 3.1): the unstratified TGV (G = 0), D3Q27, Ma 0.05, Re in
        {100, ..., 3000}: eps = -dE_k/dt (central differences) against the
        non-equilibrium eps_k in the laminar window t in [0.5, 3], and the
        peak of -dE_k/dt;
      - the Froude sweep (Sections 3.3-3.5): Re0 1600, Sc 0.7, Ma 0.1, D3Q27xD3Q19,
        Shan-Chen, Fr0 in {1, 0.1, 0.3, 0.5, 0.9, 1.5, 2.5} to t = 30: the two
        highest peaks of the total dissipation -dE_tot/dt, the peaks of R (Eq. 27)
        and Gamma, Gamma_b (Eq. 28), Fr_t (Eq. 29) and the spectral slope at t = 15;
      - the 16-bit storage rule in the double-peak regime (Fr0 = 1): FP16 and BF16
        against the FP32 run, beside an FP32 twin whose initial field differs by
        1e-6 U0 noise (the spread of the flow's own sensitivity)."""
    import numpy as np

    from paper_2605_14505_gb300 import lbm, post

    out = {"mode": "validation", "lattice": 256}
    dump = {}
    todo = set(args.validation.split(",")) if args.validation != "all" else \
        {"x1", "froude", "storage", "stencils", "resolution"}
    if "x1" in todo:
        x1 = {}
        for Re in X1_RE:
            ser, _, secs = paper_series(256, "27x19", "guo", Re, float("inf"), 1.0, X1_U0, args.x1_tend,
                                        pressure=True)
            ph = post.to_physical(ser)
            dump[f"x1_Re{int(Re)}"] = {k: v.tolist() for k, v in ph.items()}
            rate = post.total_dissipation_rate(ph["t"], ph["Ek"])
            m = (ph["t"] >= 0.5) & (ph["t"] <= 3.0)
            pk = post.peaks(ph["t"], rate, 1)
            x1[str(int(Re))] = {
                "laminar_window_balance": post.energy_balance(ph["t"], ph["Ek"], ph["eps_k"], 0.5, 3.0),
                "laminar_max_pointwise_rel_diff": float(np.max(np.abs(rate[m] / ph["eps_k"][m] - 1))),
                "peak_t": pk[0][0] if pk else None, "peak_eps": pk[0][1] if pk else None,
                "finite": bool(np.all(np.isfinite(ph["Ek"]))), "samples": len(ser), "secs": round(secs, 1)}
            print("x1", Re, x1[str(int(Re))], file=sys.stderr, flush=True)
        out["x1"] = x1
    if "froude" in todo or "storage" in todo:
        fr_out, ref_series = {}, None
        for Fr in (FROUDE if "froude" in todo else (1.0,)):
            ser, spec, secs = paper_series(PAPER["n"], PAPER["pair"], PAPER["forcing"], PAPER["Re"], Fr, PAPER["Sc"],
                                           PAPER["U0"], 30.0, spectrum_at=15.0)
            if Fr == 1.0:
                ref_series = ser
            ph = post.to_physical(ser)
            dump[f"froude_{Fr}"] = {k: v.tolist() for k, v in ph.items()}
            t = ph["t"]
            rate = post.total_dissipation_rate(t, ph["Etot"])
            R = post.buoyancy_reynolds(ph["eps_k"], PAPER["Re"], Fr)
            gam = post.flux_coefficient(ph["eps_p"], ph["eps_k"])
            rec = {"dissipation_peaks": post.peaks(t, rate, 2, separation=2.0),
                   "eps_sum_peaks": post.peaks(t, ph["eps_k"] + ph["eps_p"], 2, separation=2.0),
                   "R_peaks": post.peaks(t, R, 2, separation=2.0),
                   "Gamma_max": [float(t[np.argmax(gam[1:]) + 1]), float(np.max(gam[1:]))],
                   "Gamma_b": float(post.bulk_flux_coefficient(t, ph["eps_p"], ph["eps_k"])),
                   "Fr_t": float(post.turbulent_froude(t, ph["eps_k"], ph["Ek"], Fr)),
                   "Ek_end": float(ph["Ek"][-1]), "Ep_max": float(np.max(ph["Ep"])),
                   "finite": bool(np.all(np.isfinite(ph["Ek"]))), "samples": len(ser), "secs": round(secs, 1)}
            if spec:
                rec["spectrum_t"] = spec["t"]
                rec["spectral_slope_k4_20"] = post.spectral_slope(spec["k"], spec["E_phys"], 4, 20)
                rec["E_k_spectrum"] = [float(f"{v:.4e}") for v in spec["E_phys"][:65]]
            fr_out[str(Fr)] = rec
            print("froude", Fr, {k: v for k, v in rec.items() if k != "E_k_spectrum"}, file=sys.stderr, flush=True)
        if "froude" in todo:
            out["froude_sweep"] = fr_out
        if "storage" in todo:
            st = {}
            twin, _, _ = paper_series(PAPER["n"], PAPER["pair"], PAPER["forcing"], PAPER["Re"], 1.0, PAPER["Sc"],
                                      PAPER["U0"], 30.0, seed=7, noise_amp=1e-6)
            st["fp32_twin_1e-6"] = lbm.lbm_storage_rule(ref_series, twin, "fp32", 0.01)
            for storage in ("fp16", "bf16"):
                ser, _, secs = paper_series(PAPER["n"], PAPER["pair"], PAPER["forcing"], PAPER["Re"], 1.0, PAPER["Sc"],
                                            PAPER["U0"], 30.0, storage=storage)
                st[storage] = lbm.lbm_storage_rule(ref_series, ser, storage, 0.01)
                st[storage]["secs"] = round(secs, 1)
            out["storage_rule_fr1"] = st
            print("storage", st, file=sys.stderr, flush=True)
    if "stencils" in todo or "resolution" in todo:
        # Sections 3.2-3.3: every stencil pair at 256^3, and D3Q27xD3Q19 at 64^3 and
        # 128^3, at the paper's parameters (Fr0 = 1) to t = 30; peak heights
        # relative to the D3Q27xD3Q19 256^3 run
        runs = []
        if "stencils" in todo:
            runs += [(256, pair) for pair in ("27x19", "27x27", "19x19", "19x15", "15x7", "7x27", "19x7")]
        if "resolution" in todo:
            runs += [(64, "27x19"), (128, "27x19")] + ([] if "stencils" in todo else [(256, "27x19")])
        res, ref = {}, None
        for n, pair in runs:
            ser, _, secs = paper_series(n, pair, PAPER["forcing"], PAPER["Re"], 1.0, PAPER["Sc"], PAPER["U0"], 30.0)
            ph = post.to_physical(ser)
            dump[f"pair_{pair}_n{n}"] = {k: v.tolist() for k, v in ph.items()}
            t = ph["t"]
            rate = post.total_dissipation_rate(t, ph["Etot"])
            eps = ph["eps_k"] + ph["eps_p"]
            rec = {"dissipation_peaks": post.peaks(t, rate, 2, separation=2.0),
                   "eps_sum_peaks": post.peaks(t, eps, 2, separation=2.0),
                   "R_peaks": post.peaks(t, post.buoyancy_reynolds(ph["eps_k"], PAPER["Re"], 1.0), 2, separation=2.0),
                   "Ek_t30": float(ph["Ek"][-1]), "Ep_t30": float(ph["Ep"][-1]), "Ep_max": float(np.max(ph["Ep"])),
                   "finite": bool(np.all(np.isfinite(ph["Ek"]))), "samples": len(ser), "secs": round(secs, 1)}
            if n == 256 and pair == "27x19":
                ref = rec
            res[f"{pair}@{n}"] = rec
            print("pairs/resolution", pair, n, rec, file=sys.stderr, flush=True)
        if ref is not None:
            rp = [v for _, v in ref["eps_sum_peaks"]]
            for key, rec in res.items():
                hp = [v for _, v in rec["eps_sum_peaks"]]
                if len(hp) == len(rp) == 2:
                    rec["eps_sum_peaks_rel_to_27x19_256"] = [hp[0] / rp[0], hp[1] / rp[1]]
        out["stencils_resolution"] = res
    if args.validation_out:
        with open(args.validation_out, "w") as fh:
            json.dump(dump, fh)
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-instance batched sweep")
    ap.add_argument("--no-series", action="store_true",
                    help="skip the storage-rule series (64^3 against the stored oracle series, 256^3 workload)")
    ap.add_argument("--series-steps", type=int, default=SERIES_STEPS,
                    help="steps of the 256^3 workload series for the storage rule (0: skip it)")
    ap.add_argument("--sweep-steps", type=int, default=SWEEP_STEPS,
                    help="timed steps of the batched sweep (fewer for a bounded profiler launch list)")
    ap.add_argument("--ncu-case", choices=["fp32", "fp16", "bf16", "19x7", "19x7-fp16", "batch", "batch-step",
                                           "batch-inst"],
                    default=None,
                    help="run a small profiling case instead of the benchmark")
    ap.add_argument("--ncu-n", type=int, default=128)
    ap.add_argument("--ncu-range", action="store_true",
                    help="profiling case batch-inst: measured steps inside cudaProfilerStart/Stop")
    ap.add_argument("--ncu-steps", type=int, default=6)
    ap.add_argument("--ncu-pairing", choices=["off", "all", "even"], default="all",
                    help="profiling case: nodes per thread for 16-bit storage (lbm_set_pairing)")
    ap.add_argument("--ncu-staging", action="store_true",
                    help="profiling case: bulk-copy tile staging for 16-bit storage (lbm_set_tile_staging)")
    ap.add_argument("--validation", default=None,
                    help="run the paper's validation runs instead of the benchmark: all, or a comma list of "
                         "x1, froude, storage, stencils, resolution")
    ap.add_argument("--x1-tend", type=float, default=14.0, help="end time of the unstratified runs")
    ap.add_argument("--validation-out", default=None, help="file for the validation runs' series (paper units)")
    args = ap.parse_args()
    if args.validation:
        run_validation(args)
    elif args.ncu_case:
        run_ncu_case(args)
    elif args.impl == "reference":
        run_reference_arm(args)
    else:
        run_gpu_arm(args)


if __name__ == "__main__":
    main()
