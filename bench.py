"""Throughput of the FQNM quantised conservative step on GB300.

Workload (one bench "step" = one whole problem through the hot path):
inviscid Burgers, LF split flux (alpha = 1.3), periodic, N = 2^20 cells,
delta = 2^-16, Courant number 0.4, 10^4 time steps from the seeded
random-steps initial field:
    quantise u0 -> build and verify the transfer rule -> 10^4 steps of the
    integer update -> observable -> exact invariants.
Metric: cell updates per second (bit-exact integer states).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fqnm|reference]

N > 1 runs under torchrun: one process per GPU, each solving its own problem
(independent problems, weak scaling, no data-path collective); the time is
the maximum over ranks.  --impl reference times the CPU oracle (the plain
single-threaded implementation the tests check against) on a bounded sample
of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_06947_gb300 import inputs as I  # noqa: E402

METRIC = "cell-updates/s"
UNIT = "cell-updates/s"
BYTES_PER_UPDATE = 8          # int32 read + int32 write per cell per step
FALLBACK_HBM_GBS = 6800.0
CPU_SAMPLE_STEPS = 3000       # oracle sample: 2^20 cells x 3000 steps
REF_SAMPLE_STEPS = 100        # --impl reference: per bench step


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_problem(rank: int):
    """One independent problem per rank (weak scaling): the same workload
    shape, each rank its own seed; no data-path collective."""
    return I.burgers_problem(seed=I.BASE_SEED + 1 + rank)


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest of the ranks' values (a time): the job ends with its
    slowest rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units all ranks processed over the job's time."""
    return units_per_rank * world / seconds


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profiled_counters(kernel_tag: str, src_digest: str, workload: str = "") -> dict:
    """Per-launch counters from the committed ncu summary (profiles/traffic.txt),
    if they were taken on the current kernel sources (else {}); with
    `workload`, only a line captured on that workload."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        for line in open(path):
            if line.lstrip().startswith("#"):
                continue
            f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
            if workload and f.get("workload") != workload:
                continue
            if f.get("kernel") == kernel_tag and f.get("src_sha") == src_digest:
                return {k: float(v) for k, v in f.items()
                        if k in ("dram_bytes_per_launch", "warp_instructions_per_launch")}
    except OSError:
        pass
    return {}


def profiled_traffic(kernel_tag: str, src_digest: str):
    """DRAM bytes per launch from the committed ncu summary, or None."""
    return profiled_counters(kernel_tag, src_digest).get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch
    from paper_2604_06947_gb300 import fqnm as F
    from paper_2604_06947_gb300 import build as B

    rank, world, local = rank_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    F.load()

    p = rank_problem(rank)
    n, T = p.n, p.steps
    stream = torch.cuda.Stream()
    u0_dev = torch.from_numpy(p.u0).to(dev)
    u_out = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MB > L2

    s = F.Solver.for_problem(p, autotune=1)
    F.fqnm_set_stream(s.h, stream)
    s.n = n

    def one_step(ev=None):
        """quantise+load (rule build), T steps, observe, invariants."""
        F.fqnm_load_field(s.h, u0_dev, n, on_device=True)
        if ev is not None:
            ev[0].record(stream)
        F.fqnm_step(s.h, T)
        if ev is not None:
            ev[1].record(stream)
        F.fqnm_observe_device(s.h, u_out)
        return F.fqnm_invariants(s.h)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            inv = one_step()
    mass0 = inv["mass"][0]

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    launches0 = F.fqnm_kernel_launches()
    step_ms, region_ms = [], []
    step_launches = 0
    torch.cuda.nvtx.range_push("bench_timed")      # ncu --nvtx-include bench_timed/
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()                                   # evict L2 between steps
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ra, rb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            inv = one_step((ra, rb))
            b.record(stream)
            b.synchronize()
            step_ms.append(a.elapsed_time(b))
            region_ms.append(ra.elapsed_time(rb))
            step_launches += F.fqnm_get_stats(s.h)["launches"]   # reset by each load
            assert inv["mass"][0] == mass0, "mass not conserved"
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = F.fqnm_kernel_launches() - launches0
    stats = F.fqnm_get_stats(s.h)
    clk = clocks.stop()
    final_q = s.state()              # the last timed step's result (parity, untimed)

    total_ms = max_over_ranks(sum(step_ms), world, dev)
    value = whole_job_rate(n * T * args.steps, world, total_ms / 1e3)

    # dominant kernel: the temporal-blocked step, launched only inside the
    # stepping region; average launch duration from the events around it
    avg_launch_s = (sum(region_ms) / 1e3) / max(step_launches, 1)
    updates_per_launch = n * (T * args.steps) / max(step_launches, 1)
    kernel_tag = "k_step_tb:L%d:V%d:B%d" % (stats["layout"], stats["cells_per_thread"],
                                            stats["block"])
    counters = profiled_counters(kernel_tag, B.kernel_digest(),
                                 "burgers_lf_2^20_cells_K%d" % stats["k"])
    roofline = stepping_roofline(counters, updates_per_launch, avg_launch_s, clk, kernel_tag)

    # end to end through the C ABI with host buffers (rank-local)
    u0_host = torch.from_numpy(p.u0).pin_memory()
    u_host = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_times = []
    lib = F.load()
    for i in range(max(2, args.steps // 2) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F._check(lib.fqnm_load_field(s.h, u0_host.data_ptr(), n, 0))
        F.fqnm_step(s.h, T)
        F._check(lib.fqnm_observe(s.h, u_host.data_ptr()))
        t1 = time.perf_counter()
        if i > 0:
            e2e_times.append(t1 - t0)
    e2e_value = whole_job_rate(n * T, world,
                               max_over_ranks(statistics.median(e2e_times), world, dev))

    result = None
    if rank == 0:
        baselines = fv_baselines(F, p, stream, torch) if not args.no_fv else None
        serving = serving_block(torch) if not args.no_serving else None
        if serving is not None and world == 1 and not args.no_cpu:
            dev_s = serving.pop("_dev")
            serving["cpu_baseline"], serving["_oracle_check"] = serving_cpu_baseline(
                lambda i: dev_s.result(i).cpu().numpy(), serving.pop("_reqs"))
        elif serving is not None:
            serving.pop("_dev")
            serving.pop("_reqs")
        finals = {}
        workloads = (other_workloads(F, torch, stream, clk, finals)
                     if not args.no_workloads else None)
        cpu = cpu_baseline(p) if (world == 1 and not args.no_cpu) else None
        if cpu:
            # the CPU-baseline leg also checks the GPU's results against the
            # oracle, untimed: the timed workload's final state, the
            # high-frequency line's, and the serving stream's sampled requests
            parity = oracle_parity(p, final_q, cpu.pop("_q_sample"), finals)
            sod_accuracy(finals, workloads)
            if serving is not None:
                parity["serving_stream"] = serving.pop("_oracle_check", None)
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "burgers_lf_1m_cells_10k_steps", "n_cells": n,
                       "time_steps_per_step": T, "delta": "2^-16", "courant": 0.4,
                       "alpha": p.alpha, "flux": "burgers_lf", "boundary": "periodic",
                       "seed": I.BASE_SEED + 1, "l2": "flushed between steps (256 MB write)",
                       "parallelism": "independent problem per GPU" if world > 1 else "single GPU",
                       "plan": {"kernel": "k_step_tb", "layout": stats["layout"],
                                "cells_per_thread": stats["cells_per_thread"],
                                "block": stats["block"], "k": stats["k"],
                                "graph": stats["graph"]}},
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": 8 * n},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if cpu:
            result["cpu_baseline"] = cpu
            result["parity"] = parity
            # a compact copy inside cpu_baseline, the leg that produced it
            cpu["parity"] = {"all_equal": parity["all_equal"],
                             "checks": {k: (v.get("equal") if k != "serving_stream" else
                                            "%d/%d" % (v["requests_equal"],
                                                       v["requests_checked"]))
                                        for k, v in parity.items()
                                        if isinstance(v, dict) and v is not None}}
        if workloads and "roofline" in workloads.get("high_frequency_16m", {}):
            result["roofline"]["high_frequency_16m"] = {
                k: workloads["high_frequency_16m"]["roofline"].get(k)
                for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel",
                          "effective_hbm", "dram")}
        if baselines:
            result["fv_baseline"] = baselines
        if serving:
            result["serving"] = serving
        if workloads:
            result["workloads"] = workloads
        result["summary"] = summary(result)          # last, so a log's tail shows it
        print(json.dumps(result))
    s.close()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return result


def summary(r: dict) -> dict:
    """The headline figures of every workload in one short object."""
    w = r.get("workloads") or {}
    out = {"burgers_1m": r.get("value"), "e2e": (r.get("e2e") or {}).get("value"),
           "issue_frac": (r.get("roofline") or {}).get("frac")}
    if "high_frequency_16m" in w:
        out["high_frequency_16m"] = w["high_frequency_16m"]["value"]
    for k in ("sod_65k", "sod_1m"):
        if k in w:
            out[k] = {x: w[k].get(x) for x in ("seconds", "face_evaluations_per_s",
                                               "integer_speedup_vs_fv64", "l1_density_vs_exact",
                                               "totals_balance_exact")}
    for k in ("burgers_2d_8192", "burgers_3d_512"):
        if k in w:
            out[k] = w[k]["default"]["value"]
    sv = r.get("serving")
    if sv:
        out["serving"] = {"online": sv["batched_online"]["value"],
                          "p50_ms": sv["batched_online"]["p50_ms"],
                          "p99_ms": sv["batched_online"]["p99_ms"],
                          "offline": sv["batched_offline"]["value"],
                          "identical": sv["results_identical"]}
    fv = r.get("fv_baseline")
    if fv:
        out["fv32"] = fv["fp32"]["value"]
        out["fv64"] = fv["fp64"]["value"]
    par = r.get("parity")
    if par:
        out["parity_all_equal"] = par.get("all_equal")
    return out


def issue_peak(clk: dict):
    """Warp instructions per second the GPU can issue: 4 per SM per cycle
    (one scheduler per SM sub-partition) at the sampled SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    return 4.0 * sms * mhz * 1e6


def stepping_roofline(counters: dict, updates_per_launch: float, launch_s: float,
                      clk: dict, kernel_tag: str) -> dict:
    """The roofline of a temporal-blocked stepping kernel, against the bound
    it actually meets.

    The kernel keeps a tile in registers for K steps, so it reads and writes
    the state in HBM once per K steps: HBM is not its bound (DRAM traffic,
    from the committed ncu counters, is about 1/K of the effective bytes).
    It is bound by instruction issue on on-chip data: `achieved` is the warp
    instructions one launch executes (committed ncu count on the same
    kernel sources) over the live launch time, `peak` 4 warp instructions
    per SM per cycle at the sampled clock.  The effective-byte figure
    (8 B per cell update over the launch time, against the measured HBM copy
    peak) and the physical DRAM rate are reported beside it, named as
    such."""
    peak_hbm, peak_kind = measured_peak()
    eff_gbs = BYTES_PER_UPDATE * updates_per_launch / launch_s / 1e9
    wi = counters.get("warp_instructions_per_launch")
    traffic = counters.get("dram_bytes_per_launch")
    ipeak = issue_peak(clk)
    out = {"bound": "alu", "limiter": "instruction issue (4 warp instructions per SM "
                                      "per cycle)",
           "achieved": wi / launch_s if wi else None, "peak": ipeak,
           "unit": "warp instructions/s", "frac": (wi / launch_s / ipeak) if wi else None,
           "traffic": traffic, "kernel": kernel_tag,
           "launch_us": launch_s * 1e6, "cell_updates_per_launch": updates_per_launch,
           "warp_instructions_per_launch": wi,
           "counters": "profiles/traffic.txt (ncu, same kernel sources)" if wi else
                       "no committed counters for the current kernel sources",
           "peak_model": "4 issue slots per SM per cycle x SMs x sampled SM clock",
           "effective_hbm": {"achieved_GBps": eff_gbs, "peak_GBps": peak_hbm,
                             "peak_source": peak_kind,
                             "effective_frac_of_hbm_peak": eff_gbs / peak_hbm,
                             "bytes_model": "8 B per cell update (int32 read + write) x "
                                            "cell updates per launch; not a bandwidth: "
                                            "the state stays on chip for K steps"}}
    if traffic:
        dram_gbs = traffic / launch_s / 1e9
        out["dram"] = {"GBps": dram_gbs, "frac_of_hbm_peak": dram_gbs / peak_hbm,
                       "bytes_per_launch": traffic}
    return out


def fv_baselines(F, p, stream, torch):
    """FP32 / FP64 finite-volume baselines with the same split flux on the same
    GPU, one step per launch, and FP32 with 64 steps per launch (the integer
    kernel's temporal blocking applied to the FP scheme: the ablation that
    separates the execution strategy from the arithmetic).  Each is
    device-timed over the workload's steps (median of 5), and its L1
    distance to FQNM is taken at every checkpoint (untimed)."""
    steps, every = p.steps, 1000
    n = p.n
    q0 = F.fqnm_quantise(p.u0, p.delta)
    u0 = p.delta * q0.astype(np.float64)
    s = F.Solver.for_problem(p)
    s.load(q0)
    ref = []
    for _ in range(steps // every):
        s.step(every)
        ref.append(s.observe())
    s.close()
    out = {"time_steps": steps, "checkpoint_every": every}
    finals = {}
    for name, prec, K in (("fp32", 32, 1), ("fp64", 64, 1), ("fp32_k64", 32, 64)):
        h = F.fqnm_fv_create(F.make_flux(p.flux, alpha=p.alpha), p.dx, p.dt, "periodic", prec)
        F.fqnm_fv_set_stream(h, stream)
        F.fqnm_fv_set_k(h, K)
        F.fqnm_fv_load(h, u0)
        F.fqnm_fv_step(h, 64)
        stream.synchronize()
        runs = []
        for _ in range(5):                       # load (host copy, synchronises) untimed
            F.fqnm_fv_load(h, u0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            F.fqnm_fv_step(h, steps)
            b.record(stream)
            b.synchronize()
            runs.append(a.elapsed_time(b))
        ms = statistics.median(runs)
        F.fqnm_fv_load(h, u0)
        l1 = []
        for c in range(steps // every):
            F.fqnm_fv_step(h, every)
            u = F.fqnm_fv_observe(h, n)
            l1.append(float(p.dx * np.abs(u - ref[c]).sum()))
        finals[name] = u
        F.fqnm_fv_destroy(h)
        out[name] = {"value": n * steps / (ms / 1e3), "unit": UNIT, "steps_per_launch": K,
                     "l1_vs_fqnm": l1}
    out["fp32_k64"]["bitwise_equal_to_fp32"] = bool(np.array_equal(finals["fp32_k64"],
                                                                   finals["fp32"]))
    return out


def _timed(stream, torch, fn, reps):
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
    return statistics.median(ts)


def other_workloads(F, torch, stream, clk=None, finals=None):
    """The other workloads of the path, each timed on the device (median of
    5; the Sod runs, about 1.6 s each, once), with inputs resident on the GPU:
      - high-frequency transport, 2^24 cells, upwind nu = 0.9, 2000 steps
        (the verified closed form 9/10 replaces the table);
      - linear advection, 1024 cells, 2000 steps (a latency case);
      - Sod, 2^16 cells, componentwise-quantised Roe, to t = 0.2, and the
        FP64 Roe finite-volume baseline on the same grid."""
    from paper_2604_06947_gb300 import build as B
    peak, _ = measured_peak()
    out = {}
    for name, make in (("high_frequency_16m", I.high_frequency_problem),
                       ("linear_advection_1k", I.linear_advection_problem)):
        p = make()
        u0 = torch.from_numpy(p.u0).cuda()
        s = F.Solver.for_problem(p, autotune=1)
        F.fqnm_set_stream(s.h, stream)
        s.load_field(u0, p.n, on_device=True)
        st = F.fqnm_get_stats(s.h)

        def run():
            F.fqnm_load_field(s.h, u0, p.n, on_device=True)
            F.fqnm_step(s.h, p.steps)
        with torch.cuda.stream(stream):
            run()
            t = _timed(stream, torch, run, 5)
        F.fqnm_sync(s.h)
        launches = F.fqnm_get_stats(s.h)["launches"]      # stepping launches of one run
        if finals is not None:
            finals[name] = (p, s.state())
        rule = F.fqnm_get_rule(s.h)
        eff = BYTES_PER_UPDATE * p.n * p.steps / t / 1e9
        out[name] = {"n_cells": p.n, "time_steps": p.steps, "seconds": t,
                     "value": p.n * p.steps / t, "unit": UNIT,
                     "effective_GBps": eff, "effective_frac_of_hbm_peak": eff / peak,
                     "map": "closed form %d/%d" % (rule["num"], rule["den"])
                     if rule["evaluator"] == 2 else "table",
                     "plan": dict({k: st[k] for k in ("layout", "cells_per_thread", "block", "k")},
                                  kernel={1: "k_step_naive", 2: "k_step_tb",
                                          4: "k_step_resident"}.get(st["kernel"], st["kernel"]))}
        if name == "high_frequency_16m" and st["kernel"] == 2 and launches:
            # the large line: its own roofline object (the state, 2 x 64 MiB,
            # is about the L2's size, so HBM could bind here)
            tag = "k_step_tb:L%d:V%d:B%d" % (st["layout"], st["cells_per_thread"], st["block"])
            c = profiled_counters(tag, B.kernel_digest(),
                                  "upwind_closed_2^24_cells_K%d" % st["k"])
            out[name]["roofline"] = stepping_roofline(c, p.n * p.steps / launches,
                                                      t / launches, clk, tag)
        s.close()
    # Sod: integer Roe and the FP64 Roe FV baseline
    p = I.sod_problem(n=1 << 16)
    s = F.Solver(F.make_flux("euler_roe", gamma=p.gamma), list(p.delta), p.dx, p.dt,
                 "transmissive")
    F.fqnm_set_stream(s.h, stream)
    U0 = torch.from_numpy(p.U0.reshape(-1).copy()).cuda()
    with torch.cuda.stream(stream):
        s.load_field(U0, p.n, on_device=True)
        t_int = _timed(stream, torch, lambda: (F.fqnm_load_field(s.h, U0, p.n, on_device=True),
                                               F.fqnm_step(s.h, p.steps)), 1)
    inv = F.fqnm_invariants(s.h)
    u = s.observe()
    if finals is not None:
        # the state after the first 2000 steps (parity) and the final density
        # (its L1 error against the exact Riemann solution), both untimed
        F.fqnm_load_field(s.h, U0, p.n, on_device=True)
        F.fqnm_step(s.h, 2000)
        finals["sod_65k"] = (p, s.state().reshape(3, -1), u[0].copy())
    s.close()
    fv = F.fqnm_fv_create(F.make_flux("euler_roe", gamma=p.gamma), p.dx, p.dt, "transmissive", 64)
    F.fqnm_fv_set_stream(fv, stream)
    with torch.cuda.stream(stream):
        F.fqnm_fv_load_device(fv, U0, p.n)
        t_fv = _timed(stream, torch, lambda: (F.fqnm_fv_load_device(fv, U0, p.n),
                                              F.fqnm_fv_step(fv, p.steps)), 1)
    ufv = F.fqnm_fv_observe(fv, p.n, 3)
    F.fqnm_fv_destroy(fv)
    if finals is not None:
        finals["sod_65k_fv64"] = ufv[0].copy()
    q0 = [int(round(v)) for v in (p.U0.sum(axis=1) / np.array(p.delta))]
    out["sod_65k"] = {
        "n_cells": p.n, "time_steps": p.steps, "t_end": 0.2,
        "seconds": t_int, "face_evaluations_per_s": (p.n + 1) * p.steps / t_int,
        "fv64_roe_seconds": t_fv, "integer_speedup_vs_fv64": t_fv / t_int,
        "l1_density_vs_exact": None,             # filled in by the CPU leg (exact Riemann)
        "l1_density_fv64_vs_exact": None,
        "l1_density_integer_vs_fv64": float(p.dx * np.abs(u[0] - ufv[0]).sum()),
        "totals_balance_exact": all(inv["mass"][k] == q0[k] - inv["boundary_flux"][k]
                                    for k in range(3)),
        "bound": "FP64 unit (about 72 FP64 additions and multiplications per face; the "
                 "divisions, square roots, conversions and rounding run on the integer "
                 "pipes, FQNM_OPT_FP64 = 2)",
    }
    # the same run with every IEEE double step on the FP64 unit (FQNM_OPT_FP64 = 0)
    s = F.Solver(F.make_flux("euler_roe", gamma=p.gamma), list(p.delta), p.dx, p.dt,
                 "transmissive", fp64=0)
    F.fqnm_set_stream(s.h, stream)
    with torch.cuda.stream(stream):
        s.load_field(U0, p.n, on_device=True)
        t_fp64 = _timed(stream, torch, lambda: (F.fqnm_load_field(s.h, U0, p.n, on_device=True),
                                                F.fqnm_step(s.h, p.steps)), 1)
    same = bool(np.array_equal(s.observe(), u))
    s.close()
    out["sod_65k"]["fp64_unit_only_seconds"] = t_fp64
    out["sod_65k"]["fp64_unit_only_identical"] = same
    out["sod_1m"] = sod_large(F, torch, stream, finals)
    # Sod with the density channel alone quantised (§3.3's prototype)
    s = F.Solver(F.make_flux("euler_roe", gamma=p.gamma), list(p.delta), p.dx, p.dt,
                 "transmissive", quantise_mask=1)
    F.fqnm_set_stream(s.h, stream)
    with torch.cuda.stream(stream):
        s.load_field(U0, p.n, on_device=True)
        t_rho = _timed(stream, torch, lambda: (F.fqnm_load_field(s.h, U0, p.n, on_device=True),
                                               F.fqnm_step(s.h, p.steps)), 1)
    inv1 = F.fqnm_invariants(s.h)
    u1 = s.observe()
    s.close()
    out["sod_65k_density_only"] = {
        "n_cells": p.n, "time_steps": p.steps, "seconds": t_rho,
        "quantised": "rho (m, E in double with the same Roe flux)",
        "l1_density_vs_componentwise": float(p.dx * np.abs(u1[0] - u[0]).sum()),
        "l1_density_vs_fv64": float(p.dx * np.abs(u1[0] - ufv[0]).sum()),
        "density_balance_exact": inv1["mass"][0] == q0[0] - inv1["boundary_flux"][0],
    }
    out["burgers_2d_4096"] = nd_workload(F, torch, stream, (4096, 4096), 240)
    out["burgers_2d_8192"] = nd_workload(F, torch, stream, (8192, 8192), 48)
    out["burgers_3d_256"] = nd_workload(F, torch, stream, (256, 256, 256), 96)
    out["burgers_3d_512"] = nd_workload(F, torch, stream, (512, 512, 512), 24)
    out["burgers_sine_convergence"] = convergence_sweep(F, torch, stream)
    out["level_statistics_1m"] = level_statistics(F, torch, stream)
    return out


def sod_large(F, torch, stream, finals, n=1 << 20, window=20_000):
    """Sod on 2^20 cells: the integer Roe step against the FP64 Roe FV
    baseline over the first 20,000 steps (device-timed), and the whole run
    to t = 0.2 (919,210 steps, device-timed, once) with the exact balance of
    all three totals; the L1 density error against the exact Riemann solution
    and the full-state parity of the first 2000 steps are added by the CPU
    leg."""
    p = I.sod_problem(n=n)
    U0 = torch.from_numpy(p.U0.reshape(-1).copy()).cuda()
    s = F.Solver(F.make_flux("euler_roe", gamma=p.gamma), list(p.delta), p.dx, p.dt,
                 "transmissive")
    F.fqnm_set_stream(s.h, stream)
    with torch.cuda.stream(stream):
        s.load_field(U0, p.n, on_device=True)
        t_int = _timed(stream, torch, lambda: (F.fqnm_load_field(s.h, U0, p.n, on_device=True),
                                               F.fqnm_step(s.h, window)), 1)
        if finals is not None:
            F.fqnm_load_field(s.h, U0, p.n, on_device=True)
            F.fqnm_step(s.h, 2000)
            finals["sod_1m_2000"] = (p, s.state().reshape(3, -1))
        t_full = _timed(stream, torch, lambda: (F.fqnm_load_field(s.h, U0, p.n, on_device=True),
                                                F.fqnm_step(s.h, p.steps)), 1)
    inv = F.fqnm_invariants(s.h)
    u = s.observe()
    s.close()
    fv = F.fqnm_fv_create(F.make_flux("euler_roe", gamma=p.gamma), p.dx, p.dt, "transmissive", 64)
    F.fqnm_fv_set_stream(fv, stream)
    with torch.cuda.stream(stream):
        F.fqnm_fv_load_device(fv, U0, p.n)
        t_fv = _timed(stream, torch, lambda: (F.fqnm_fv_load_device(fv, U0, p.n),
                                              F.fqnm_fv_step(fv, window)), 1)
    F.fqnm_fv_destroy(fv)
    q0 = [int(round(v)) for v in (p.U0.sum(axis=1) / np.array(p.delta))]
    if finals is not None:
        finals["sod_1m_rho"] = (p, u[0].copy())
    return {"n_cells": p.n, "time_steps": p.steps, "t_end": 0.2,
            "seconds": t_full, "face_evaluations_per_s": (p.n + 1) * p.steps / t_full,
            "first_steps": window, "first_steps_seconds": t_int,
            "fv64_roe_first_steps_seconds": t_fv, "integer_speedup_vs_fv64": t_fv / t_int,
            "totals_balance_exact": all(inv["mass"][k] == q0[k] - inv["boundary_flux"][k]
                                        for k in range(3)),
            "l1_density_vs_exact": None}


def nd_workload(F, torch, stream, dims, steps):
    """Burgers on a periodic 2-D or 3-D grid (directional composition):
    device-timed steps, the default plan (2-D: the walk at K = 4; 3-D: the
    one-step streaming kernel), the autotuned plan, other plans and the
    two-word (unpacked) map table."""
    p = I.burgers_nd_problem(dims, steps=steps)
    u0 = torch.from_numpy(p.u0).cuda()
    out = {"dims": list(dims), "n_cells": p.n, "time_steps": steps}
    plans = [("default", {}), ("autotuned", {"autotune": 1})] + (
        [("tile_64x32", {"nd_tile": 3}), ("one_step", {"kernel": 1}),
         ("two_word_table", {"pack16": 0})] if len(dims) == 2 else
        [("walk_k1", {"k": 1}), ("walk_k2", {"k": 2}), ("walk_k3", {"k": 3}),
         ("two_word_table", {"pack16": 0})])
    for name, opt in plans:
        s = F.Solver.for_problem(p, **opt)
        s.set_grid(p.dims)
        F.fqnm_set_stream(s.h, stream)
        with torch.cuda.stream(stream):
            s.load_field(u0, p.n, on_device=True)
            m0 = F.fqnm_invariants(s.h)["mass"][0]
            t = _timed(stream, torch, lambda: F.fqnm_step(s.h, steps), 5)
        inv = F.fqnm_invariants(s.h)
        st = F.fqnm_get_stats(s.h)
        s.close()
        out[name] = {"seconds": t, "value": p.n * steps / t, "unit": UNIT,
                     "effective_GBps": BYTES_PER_UPDATE * p.n * steps / t / 1e9,
                     "mass_exact": inv["mass"][0] == m0,
                     "plan": {"kernel": {1: "one step", 5: "walk", 6: "register tile"}.get(
                         st["kernel"], st["kernel"]), "nd_tile": st["layout"], "k": st["k"]}}
    return out


def convergence_sweep(F, torch, stream, kmax: int = 14):
    """The paper's Burgers data (u0 = 0.5 + sin 2 pi x) to t = 0.3 on
    N = 2^7 .. 2^kmax cells with delta = dx^(3/2) (delta/dx -> 0), against the
    Hopf-Lax entropy solution on 16 N candidates per period, both on the GPU.
    Also times the Hopf-Lax kernel (FP64-bound: 4 FP64 operations per
    evaluation; the compare runs on the integer pipe) on the largest grid."""
    import math
    rows, hl = [], {}
    for k in range(7, kmax + 1):
        n = 1 << k
        p = I.burgers_sine_problem(n=n, delta=2.0 ** -math.ceil(1.5 * k))
        s = F.Solver.for_problem(p)
        F.fqnm_set_stream(s.h, stream)
        u0 = torch.from_numpy(p.u0).cuda()
        with torch.cuda.stream(stream):
            t = _timed(stream, torch, lambda: (F.fqnm_load_field(s.h, u0, n, on_device=True),
                                               F.fqnm_step(s.h, p.steps)), 1)
        u = s.observe()
        s.close()
        x = I.cell_centres(n)
        y, U = I.sine_candidates(16 * n)
        dx_, dy, dU = (torch.from_numpy(a).cuda() for a in (x, y, U))
        du = torch.empty(n, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            th = _timed(stream, torch, lambda: F.fqnm_hopf_lax(dx_, dy, dU, 0.3, nx=n, ny=y.size,
                                                               u=du, stream=stream), 5)
        ue = du.cpu().numpy()
        rows.append({"n_cells": n, "delta": p.delta, "time_steps": p.steps, "seconds": t,
                     "l1_vs_hopf_lax": float(p.dx * np.abs(u - ue).sum())})
        hl = {"n_points": n, "n_candidates": int(y.size), "seconds": th,
              "evaluations_per_s": n * y.size / th}
    e = np.array([r["l1_vs_hopf_lax"] for r in rows])
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    fp64_peak = 2.0 * sm * 2.07e9                      # FP64 ops/s: 2 per SM per clock
    hl["fp64_ops_per_s"] = 4 * hl["evaluations_per_s"]
    hl["fp64_peak_ops_per_s"] = fp64_peak
    hl["frac_of_fp64_peak"] = hl["fp64_ops_per_s"] / fp64_peak
    return {"t_end": 0.3, "delta": "dx^(3/2)", "rows": rows,
            "rates": [float(r) for r in np.log2(e[:-1] / e[1:])], "hopf_lax": hl}


def level_statistics(F, torch, stream):
    """One level-statistics record (histograms, entropy, row-sum defect,
    sorted transition matrix) on the Burgers 2^20-cell workload after 300
    steps, against one plain step."""
    p = I.burgers_problem()
    s = F.Solver.for_problem(p)
    F.fqnm_set_stream(s.h, stream)
    u0 = torch.from_numpy(p.u0).cuda()
    s.load_field(u0, p.n, on_device=True)
    s.step(300)
    rec = s.level_step()                               # grows the work buffers
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        rec = s.level_step()
    t_rec = (time.perf_counter() - t0) / reps
    F.fqnm_sync(s.h)
    t0 = time.perf_counter()
    for _ in range(reps):
        F.fqnm_step(s.h, 1)
        F.fqnm_sync(s.h)
    t_step = (time.perf_counter() - t0) / reps
    s.close()
    return {"n_cells": p.n, "seconds_per_record": t_rec, "seconds_per_plain_step": t_step,
            "record": {k: rec[k] for k in ("step", "occupied", "S", "n_eff", "rho", "pairs",
                                           "moved")}}


def serving_block(torch):
    """The batched serving path on the 4096-request stream (Poisson arrivals
    at 2000/s, half linear advection, half Burgers, N log-uniform in
    [256, 2^20], steps log-uniform in [100, 10^4]): online latencies and
    throughput with the plan tuned online, the same requests all at once
    (offline), and one problem at a time through the single-problem path."""
    from paper_2604_06947_gb300 import serve as S
    reqs = I.serving_stream()
    dev = S.DeviceStream(reqs)
    online = S.serve_batched(reqs, dev=dev, plan="autotune")
    out_online = dev.out.clone()                 # the online pass's results, kept
    tuned = {k: online["plan"][k] for k in ("cells_per_thread", "block", "k", "layout")}
    offline_reqs = [I.ServeRequest(r.rid, 0.0, r.problem, r.data_seed) for r in reqs]
    offline = S.serve_batched(offline_reqs, dev=dev, plan=tuned)
    out_single = torch.empty_like(dev.out)
    one = S.serve_one_by_one(reqs, dev=dev, out=out_single)
    online_identical = bool(torch.equal(out_single, out_online))
    offline_identical = bool(torch.equal(out_single, dev.out))
    dev.out.copy_(out_online)                    # the oracle check reads the online results
    keys = ("value", "p50_ms", "p99_ms", "max_ms")
    return {
        "workload": "4096 requests, Poisson 2000/s, half linear / half Burgers, "
                    "N log-uniform [256, 2^20], steps log-uniform [100, 10^4], int32, delta 2^-16",
        "cell_updates": online["cell_updates"],
        "batched_online": dict({k: online[k] for k in keys}, makespan_s=online["makespan_s"],
                               gpu_value=online["value_gpu"], epochs=online["epochs"],
                               plan=tuned),
        "batched_offline": {"value": offline["value"], "gpu_value": offline["value_gpu"],
                            "makespan_s": offline["makespan_s"]},
        "one_problem_at_a_time": dict({k: one[k] for k in keys}, busy_s=one["busy_s"]),
        "online_identical_to_one_at_a_time": online_identical,
        "offline_identical_to_one_at_a_time": offline_identical,
        "results_identical": online_identical and offline_identical,
        "unit": UNIT,
        "_dev": dev, "_reqs": reqs,
    }


# ---------------------------------------------------------------------------
# CPU oracle
# ---------------------------------------------------------------------------

def host_cpu() -> dict:
    """The host's CPU model and core count, as the OS reports them."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return {"cpu_model": model or platform.processor() or "unknown",
            "machine": platform.machine(), "nproc": os.cpu_count()}


def cpu_baseline(p, steps: int = CPU_SAMPLE_STEPS):
    from oracle import oracle as O
    q0 = O.quantise(p.u0, p.delta)
    t0 = time.perf_counter()
    q = O.step(q0, p.flux, p.delta, p.dx, p.dt, steps, alpha=p.alpha)
    dt = time.perf_counter() - t0
    return {"value": p.n * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d cells x %d of the 10^4 time steps (same seeded problem), "
                      "single-threaded C oracle, %.1f s" % (p.n, steps, dt),
            "host": host_cpu(), "_q_sample": (steps, q)}


def oracle_parity(p, final_q, sample, finals) -> dict:
    """The GPU's results against the oracle, element by element (untimed).

    - the timed workload: the final state of the last timed bench step
      (2^20 cells after 10^4 steps) against the oracle's, assembled from
      dependency windows run in parallel host processes; and the state
      after the CPU baseline's own sample of steps against that sample;
    - the high-frequency line (2^24 cells, 2000 steps): the whole final
      state, the same way;
    - the serving stream's sampled requests (filled in by the serving leg)."""
    import torch
    from oracle import oracle as O
    from paper_2604_06947_gb300 import fqnm as F
    out = {}
    t0 = time.perf_counter()
    q0 = O.quantise(p.u0, p.delta)
    want = O.step_by_windows(q0, p.steps, p.flux, p.delta, p.dx, p.dt, alpha=p.alpha)
    diff = int((final_q.astype(np.int64) != want).sum())
    out["burgers_1m_10k_steps"] = {"cells": int(p.n), "time_steps": p.steps,
                                   "cells_differing": diff, "equal": diff == 0,
                                   "oracle": "full state from dependency windows, %d host "
                                             "processes, %.1f s"
                                             % (os.cpu_count() or 1,
                                                time.perf_counter() - t0)}
    steps, q_cpu = sample
    s = F.Solver.for_problem(p)
    s.load(F.fqnm_quantise(p.u0, p.delta)).step(steps)
    diff = int((s.state().astype(np.int64) != q_cpu).sum())
    s.close()
    out["burgers_1m_cpu_sample"] = {"cells": int(p.n), "time_steps": steps,
                                    "cells_differing": diff, "equal": diff == 0,
                                    "oracle": "the CPU baseline's own single-threaded run"}
    if "high_frequency_16m" in finals:
        ph, qh = finals["high_frequency_16m"]
        t0 = time.perf_counter()
        want = O.step_by_windows(O.quantise(ph.u0, ph.delta), ph.steps, ph.flux, ph.delta,
                                 ph.dx, ph.dt, a=ph.a)
        diff = int((qh.astype(np.int64) != want).sum())
        out["high_frequency_16m_2000_steps"] = {
            "cells": int(ph.n), "time_steps": ph.steps, "cells_differing": diff,
            "equal": diff == 0,
            "oracle": "full state from dependency windows, %d host processes, %.1f s"
                      % (os.cpu_count() or 1, time.perf_counter() - t0)}
    if "sod_65k" in finals:
        ps, q2000, _ = finals["sod_65k"]
        q0s = np.stack([O.quantise(ps.U0[k], ps.delta[k]) for k in range(3)]).astype(np.int64)
        want = O.euler_step_by_windows(q0s, 2000, ps.gamma, ps.delta, ps.dx, ps.dt)
        diff = int((q2000 != want).any(axis=0).sum())
        out["sod_65k_2000_steps"] = {"cells": int(ps.n), "time_steps": 2000,
                                     "cells_differing": diff, "equal": diff == 0,
                                     "oracle": "full state (rho, m, E) from dependency "
                                               "windows"}
    if "sod_1m_2000" in finals:
        ps, q2000 = finals["sod_1m_2000"]
        t0 = time.perf_counter()
        q0s = np.stack([O.quantise(ps.U0[k], ps.delta[k]) for k in range(3)]).astype(np.int64)
        want = O.euler_step_by_windows(q0s, 2000, ps.gamma, ps.delta, ps.dx, ps.dt)
        diff = int((q2000 != want).any(axis=0).sum())
        out["sod_1m_2000_steps"] = {"cells": int(ps.n), "time_steps": 2000,
                                    "cells_differing": diff, "equal": diff == 0,
                                    "oracle": "full state (rho, m, E) from dependency windows, "
                                              "%d host processes, %.1f s"
                                              % (os.cpu_count() or 1, time.perf_counter() - t0)}
    out["all_equal"] = all(v.get("equal", False) for v in out.values() if isinstance(v, dict))
    return out


def sod_accuracy(finals, workloads):
    """L1 density error of the Sod runs against the exact Riemann solution
    at t = 0.2 (the oracle's exact solver, sampled at the cell centres)."""
    from oracle import oracle as O
    if not workloads or "sod_65k" not in finals or "sod_65k" not in workloads:
        return
    p, _, rho = finals["sod_65k"]
    x = I.cell_centres(p.n)
    rex, _, _ = O.riemann_sample(p.gamma, I.SOD_LEFT, I.SOD_RIGHT, 0.5, I.SOD_T_END, x)
    workloads["sod_65k"]["l1_density_vs_exact"] = float(p.dx * np.abs(rho - rex).sum())
    if "sod_65k_fv64" in finals:
        workloads["sod_65k"]["l1_density_fv64_vs_exact"] = float(
            p.dx * np.abs(finals["sod_65k_fv64"] - rex).sum())
    if "sod_1m_rho" in finals and "sod_1m" in workloads:
        p, rho = finals["sod_1m_rho"]
        x = I.cell_centres(p.n)
        rex, _, _ = O.riemann_sample(p.gamma, I.SOD_LEFT, I.SOD_RIGHT, 0.5, I.SOD_T_END, x)
        workloads["sod_1m"]["l1_density_vs_exact"] = float(p.dx * np.abs(rho - rex).sum())


def _oracle_request(job):
    """One serving request solved by the single-threaded oracle (a pool
    worker): returns its index, cell updates, the seconds of its steps and
    its final state."""
    from oracle import oracle as O
    i, rq = job
    p = I.materialise(rq)
    q0 = O.quantise(p.u0, p.delta)
    p.u0 = None
    t0 = time.perf_counter()
    q = O.step(q0, p.flux, p.delta, p.dx, p.dt, p.steps, a=p.a, alpha=p.alpha)
    return i, p.n * p.steps, time.perf_counter() - t0, q


def serving_cpu_baseline(result_of, reqs, every: int = 16):
    """The serving stream's problems on the host cores: one single-threaded
    oracle instance per core (a spawned process pool), on every 16th request
    of the 4096; value = their cell updates / the pool's wall time.  Each
    oracle result is then compared, element by element, with the online
    batched pass's result for that request (result_of(i), an int array)."""
    import multiprocessing as mp
    idx = list(range(0, len(reqs), every))
    cores = os.cpu_count() or 1
    order = sorted(idx, key=lambda i: -reqs[i].problem.n * reqs[i].problem.steps)
    jobs = [(i, reqs[i]) for i in order]
    with mp.get_context("spawn").Pool(cores) as pool:
        t0 = time.perf_counter()
        res = pool.map(_oracle_request, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    updates = sum(r[1] for r in res)
    equal = sum(int(np.array_equal(np.asarray(result_of(i), dtype=np.int64), q))
                for i, _, _, q in res)
    base = {"value": updates / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "every %dth request (%d of 4096, %.3g cell updates), one single-threaded "
                      "C oracle per core, %.1f s wall, %.1f core-s"
                      % (every, len(idx), updates, wall, sum(r[2] for r in res))}
    check = {"requests_checked": len(res), "requests_equal": equal,
             "equal": equal == len(res),
             "compared": "online batched result vs the oracle, every %dth request" % every}
    return base, check


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return None
    from oracle import oracle as O
    p = I.burgers_problem()
    q0 = O.quantise(p.u0, p.delta)
    for _ in range(args.warmup):
        O.step(q0, p.flux, p.delta, p.dx, p.dt, 10, alpha=p.alpha)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.step(q0, p.flux, p.delta, p.dx, p.dt, REF_SAMPLE_STEPS, alpha=p.alpha)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = p.n * REF_SAMPLE_STEPS * args.steps / total
    res = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "burgers_lf_1m_cells_10k_steps", "n_cells": p.n,
                   "time_steps_per_step": REF_SAMPLE_STEPS,
                   "note": "each step is a bounded sample (%d of the 10^4 time steps)"
                           % REF_SAMPLE_STEPS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d cells x %d time steps per bench step"
                                   % (p.n, REF_SAMPLE_STEPS), "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(res))
    return res


def run_sod_full(args):
    """Sod on 2^m cells to t = 0.2 on one GPU, device-timed as one run with
    the SM clocks sampled: the integer Roe step's full run, the exact balance
    of all three totals against the counted boundary transfer, the L1
    density error against the exact Riemann solution, and (CPU leg) the
    whole state after the first 2000 steps against the oracle."""
    import torch
    from paper_2604_06947_gb300 import fqnm as F
    torch.cuda.set_device(0)
    F.load()
    p = I.sod_problem(n=1 << args.sod_full)
    stream = torch.cuda.Stream()
    U0 = torch.from_numpy(p.U0.reshape(-1).copy()).cuda()
    s = F.Solver(F.make_flux("euler_roe", gamma=p.gamma), list(p.delta), p.dx, p.dt,
                 "transmissive")
    F.fqnm_set_stream(s.h, stream)
    with torch.cuda.stream(stream):
        s.load_field(U0, p.n, on_device=True)
        F.fqnm_step(s.h, 2000)
        q2000 = s.state().reshape(3, -1)
        F.fqnm_load_field(s.h, U0, p.n, on_device=True)
        stream.synchronize()
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        F.fqnm_step(s.h, p.steps)
        b.record(stream)
        b.synchronize()
        clk = clocks.stop()
    secs = a.elapsed_time(b) / 1e3
    inv = F.fqnm_invariants(s.h)
    u = s.observe()
    s.close()
    q0 = [int(round(v)) for v in (p.U0.sum(axis=1) / np.array(p.delta))]
    res = {"workload": "sod_%d_cells_to_t0.2" % p.n, "n_cells": p.n, "time_steps": p.steps,
           "seconds": secs, "face_evaluations_per_s": (p.n + 1) * p.steps / secs,
           "totals_balance_exact": all(inv["mass"][k] == q0[k] - inv["boundary_flux"][k]
                                       for k in range(3)),
           "boundary_transfer": inv["boundary_flux"], "clocks": clk}
    if not args.no_cpu:
        from oracle import oracle as O
        x = I.cell_centres(p.n)
        rex, _, _ = O.riemann_sample(p.gamma, I.SOD_LEFT, I.SOD_RIGHT, 0.5, I.SOD_T_END, x)
        res["l1_density_vs_exact"] = float(p.dx * np.abs(u[0] - rex).sum())
        qs = np.stack([O.quantise(p.U0[k], p.delta[k]) for k in range(3)]).astype(np.int64)
        want = O.euler_step_by_windows(qs, 2000, p.gamma, p.delta, p.dx, p.dt)
        diff = int((q2000 != want).any(axis=0).sum())
        res["parity_first_2000_steps"] = {"cells_differing": diff, "equal": diff == 0}
    print(json.dumps(res))
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fqnm", choices=["fqnm", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fv", action="store_true", help="skip the FP finite-volume baseline")
    ap.add_argument("--no-serving", action="store_true", help="skip the batched serving stream")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the other workloads (high-frequency 16M, linear 1k, Sod)")
    ap.add_argument("--sod-full", type=int, default=0, metavar="M",
                    help="only run Sod on 2^M cells to t = 0.2 and print its record")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.sod_full:
        run_sod_full(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
