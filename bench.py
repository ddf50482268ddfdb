"""Benchmark of the RBE2D k-space force on GB300.

Workload (one "step"): draw the batch (P = 500) and evaluate the random-batch k-space
force with the image series folded into per-k coefficients, for N = 1e6 charges in a
200 x 200 x 20 slab with gamma_top = 0.9, gamma_bot = -0.9 (M = 14, Lz = 594).  Metric:
particle-evals/s = N / (time of one force evaluation), FP32-mixed mode; the FP64 mode
of the same library is timed beside it.

Timed region: inputs resident in HBM; L2 is flushed (512 MB memset + 256 MB read) before every timed
step, outside the step's CUDA events.  With --gpus N > 1 under torchrun every rank runs
its own independent replica (weak scaling; the path has no cross-rank exchange here).

--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the
same workload (a subset of the P wave vectors, scaled to the full batch).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "slab_n1e6"
METRIC = "RBE2D force particle-evals/s at N=1e6,P=500 (FP32 vs FP64 GPU) at 1e-4 err"
UNIT = "particle-evals/s"
SMS = 152
MUFU_PER_CLK_SM = 16      # sin/cos results per clock per SM (CUDA throughput table; measured 16.0 on GB300)
SM_MAX_MHZ = 2070.0
MD_SKIN = 0.3             # Verlet skin of the MD leg's real-space pair lists


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _parallelism(ws):
    return f"replicas x{ws}" if ws > 1 else "single GPU"


def _workload_config(w, ws=1):
    cfg = {"workload": w.name, "N": w.N, "P": w.P, "Lx": w.Lx, "Ly": w.Ly, "H": w.H,
           "gamma_top": w.gamma_top, "gamma_bot": w.gamma_bot, "M": w.M, "Lz": w.Lz,
           "alpha": round(w.alpha, 6), "charges": "+1/-1 neutral, uniform positions (seed 1)",
           "k_batch": "Philox4x64-10 i.i.d. from exp(-k^2/4a^2)/S, key=seed 0, counter=(l,attempt,step,0)",
           "l2": "flushed before every timed step (512 MB memset, then a 256 MB read so the cache holds "
                 "no dirty lines; both outside the step events)",
           "parallelism": _parallelism(ws)}
    return cfg


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, gpu_index):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"rbe2d_bench_clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0])); mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2405_06333_gb300 import binding as B
    from paper_2405_06333_gb300.rbe2d import RBE2D
    from paper_2405_06333_gb300.synthetic import WORKLOADS, workload_inputs

    ws, rank, local = _dist()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    w = WORKLOADS[args.workload]
    if args.md_only:  # profiling runs of the MD step
        print(json.dumps({"md": md_leg(w, dev, args.md_steps)}))
        return
    if args.batch_only:  # profiling runs of the batched launch
        print(json.dumps({"batched": batch_leg(dev, args.batch_steps, args.batch_tuning),
                          "probe": B.rbe2d_pipe_probe()}))
        return
    pos_h, q_h = workload_inputs(w)
    pos = torch.as_tensor(pos_h, device=dev)
    q = torch.as_tensor(q_h, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sweep = torch.zeros(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sink = torch.empty((), dtype=torch.float32, device=dev)

    def flush_l2():
        # overwrite a buffer 4x the L2, then read another 2x the L2: the step starts with
        # a cold cache that holds clean lines, so it pays no write-back of the flush
        flush.zero_()
        torch.sum(sweep, 0, out=sink)

    if args.adjoint_only:  # profiling runs of the energy adjoint (both tuners, then the timed steps)
        print(json.dumps({"adjoint": adjoint_leg(dev, flush_l2, max(3, min(args.steps, 20)))}))
        return

    def make(prec):
        return RBE2D(w.Lx, w.Ly, w.H, n_max=w.N, P=w.P, gamma_top=w.gamma_top, gamma_bot=w.gamma_bot, M=w.M,
                     Lz=w.Lz, alpha=w.alpha, r_c=w.r_c, seed=w.seed, precision=prec)

    def timed(model, steps, warmup, step0=0):
        """Per step: flush L2, then [sample | structure factor | force] with events."""
        st = torch.cuda.current_stream(dev)
        F = torch.empty((w.N, 3), dtype=model.out_dtype, device=dev)
        nflags = B.RBE2D_KSPACE | B.RBE2D_IBC
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        for i in range(warmup):
            B.rbe2d_sample_k(model.ctx, step0 + i, None)
            B.rbe2d_force(model.ctx, w.N, pos, q, nflags, F, None, None)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(dev.index) if rank == 0 else None
        # per-kernel events on the library's stream, around the two dominant kernels only
        B.rbe2d_timer_enable(model.ctx, steps, ("structure_factor", "force"))
        launches0 = B.rbe2d_kernel_launches()
        t0 = time.perf_counter()
        for i in range(steps):
            flush_l2()
            ev[i][0].record(st)
            B.rbe2d_sample_k(model.ctx, step0 + warmup + i, None)
            B.rbe2d_structure_factor(model.ctx, w.N, pos, q, 0, None)
            ev[i][1].record(st)
            B.rbe2d_force(model.ctx, w.N, pos, q, nflags | B.RBE2D_REUSE_SF, F, None, None)
            ev[i][2].record(st)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = clk.stop() if clk else None
        launches = B.rbe2d_kernel_launches() - launches0  # this library's kernels in the timed steps
        kt = B.rbe2d_timer_read(model.ctx)
        B.rbe2d_timer_enable(model.ctx, 0)
        kernel_ms = {k: ms / n for k, (ms, n) in kt.items() if n > 0}
        step_ms = [ev[i][0].elapsed_time(ev[i][2]) for i in range(steps)]
        sf_ms = [ev[i][0].elapsed_time(ev[i][1]) for i in range(steps)]
        force_ms = [ev[i][1].elapsed_time(ev[i][2]) for i in range(steps)]
        model.sync_status()
        return {"step_ms": float(np.mean(step_ms)), "sf_ms": float(np.mean(sf_ms)),
                "force_ms": float(np.mean(force_ms)), "wall_s": wall, "clocks": clocks, "F": F,
                "kernel_ms": kernel_ms, "launches": launches}

    m32 = make("fp32")
    # project autotuner: FMA-pipe share of the sin/cos and launch shape of each FP32 kernel
    B.rbe2d_sample_k(m32.ctx, 0, None)
    if args.tuning:  # profiler runs: a fixed choice instead of timing under the profiler
        t = [int(x) for x in args.tuning.split(",")]
        B.rbe2d_set_tuning(m32.ctx, *t)
        tuning = {"sf_poly": t[0], "force_poly": t[1], "sf_shape": t[2], "force_shape": t[3], "set": True}
    else:
        tuning = B.rbe2d_autotune(m32.ctx, w.N, pos, q, B.RBE2D_IBC, torch.empty((w.N, 3), device=dev))
    r32 = timed(m32, args.steps, args.warmup)
    # max over ranks of the per-step time
    t_step = torch.tensor([r32["step_ms"]], device=dev, dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(t_step, op=dist.ReduceOp.MAX)
    t_step = float(t_step.item())
    if args.quick:  # profiling runs: the FP32 path only
        if rank == 0:
            print(json.dumps({"quick": True, "ms_per_step": t_step, "phases_ms": [r32["sf_ms"], r32["force_ms"]],
                              "kernel_ms": r32["kernel_ms"],
                              "tuning": tuning}))
        m32.close()
        if ws > 1:
            dist.destroy_process_group()
        return

    # FP64 mode of the same library on the same batch (speedup denominator), fewer steps
    m64 = make("fp64")
    r64 = timed(m64, max(2, min(args.steps, 3)), 1)
    # FP32 vs FP64-GPU error on the same batch (step 0)
    B.rbe2d_sample_k(m32.ctx, 0, None)
    B.rbe2d_sample_k(m64.ctx, 0, None)
    F32 = m32.force(pos, q)
    F64 = m64.force(pos, q)
    err = float(torch.linalg.norm((F32.double() - F64)) / torch.linalg.norm(F64))

    # e2e: the same C entry point with HOST buffers (pinned), copies inside the timed region
    pos_pin = torch.as_tensor(pos_h).pin_memory()
    q_pin = torch.as_tensor(q_h).pin_memory()
    F_pin = torch.empty((w.N, 3), dtype=torch.float32).pin_memory()
    e_pin = torch.empty(4, dtype=torch.float64).pin_memory()
    hflags = B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_ENERGY | B.RBE2D_HOST_BUFFERS
    for i in range(2):
        B.rbe2d_sample_k(m32.ctx, i, None)
        B.rbe2d_force(m32.ctx, w.N, pos_pin, q_pin, hflags, F_pin, None, e_pin)
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.steps, 30))
    t_calls = []
    for i in range(e2e_steps):
        # the same cache state as the device-timed steps: L2 flushed before every call,
        # outside the timed call (the call itself synchronises before it returns)
        flush_l2()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.rbe2d_sample_k(m32.ctx, 100 + i, None)
        B.rbe2d_force(m32.ctx, w.N, pos_pin, q_pin, hflags, F_pin, None, e_pin)
        t_calls.append(time.perf_counter() - t0)
    t_e2e = float(np.mean(t_calls))
    t_e2e_t = torch.tensor([t_e2e], device=dev, dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(t_e2e_t, op=dist.ReduceOp.MAX)
    t_e2e = float(t_e2e_t.item())

    # adjoint leg (energy backward) and the other workloads, FP32-mixed and FP64 modes
    adjoint_out = workloads_out = None
    if not args.no_extra:
        adjoint_out = adjoint_leg(dev, flush_l2, max(3, min(args.steps, 20)))
        workloads_out = workloads_leg(dev, flush_l2, max(3, min(args.steps, 20)))

    # batched leg: 512 independent slabs in one persistent launch (autotuned)
    batch_out = None
    if not args.no_batch:
        batch_out = batch_leg(dev, max(3, min(args.steps, 50)))

    # MD leg: Langevin BAOAB steps (k-space + IBC + real space + WCA + walls) replayed
    # from a captured CUDA graph, 1000 steps
    md_out = None
    if not args.no_md:
        md_out = md_leg(w, dev, args.md_steps)
        if not args.no_extra:
            md_out["heating"] = md_heating(w, dev, 2 * args.md_steps)

    # measured per-clock throughput of the MUFU, FP32 and FP64 pipes (the derived peak's
    # unit counts, checked on this device)
    probe = B.rbe2d_pipe_probe()

    # roofline of the dominant kernel: sin/cos results (MUFU) per second
    diel = 1 if (w.M > 0 and (w.gamma_top != 0 or w.gamma_bot != 0)) else 0
    sincos_per_pair = 2 * (2 if diel else 1)  # sin and cos of theta1 (and theta2)
    mufu_ops = w.N * w.P * sincos_per_pair
    peak = MUFU_PER_CLK_SM * SMS * SM_MAX_MHZ * 1e6
    # each kernel's mean launch duration from the library's own events over the timed steps
    k_sf, k_force = r32["kernel_ms"]["structure_factor"], r32["kernel_ms"]["force"]
    dominant = "sf" if k_sf >= k_force else "force"
    dur = max(k_sf, k_force) * 1e-3
    achieved = mufu_ops / dur
    other = min(k_sf, k_force) * 1e-3

    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            import hashlib
            ent = json.load(open(prof))[dominant]
            src = b"".join(open(os.path.join(ROOT, f), "rb").read() for f in ent["sources"])
            if hashlib.sha256(src).hexdigest()[:16] == ent["sources_sha256_16"]:
                traffic = ent["bytes"]  # counters taken on this exact kernel source
        except Exception:
            traffic = None

    value = ws * w.N / (t_step * 1e-3)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (phases, products) + f64 (reductions, coefficients)", "data": "synthetic",
        "config": _workload_config(w, ws),
        "fp64_mode": {"value": ws * w.N / (r64["step_ms"] * 1e-3), "ms_per_step": r64["step_ms"],
                      "speedup_fp32_over_fp64": r64["step_ms"] / t_step},
        "rel_l2_fp32_vs_fp64_gpu": err,
        "pair_evals_per_s": value * w.P,
        "phases_ms": {"sample+structure_factor(with packing)+fold": r32["sf_ms"], "force": r32["force_ms"]},
        "kernel_ms": r32["kernel_ms"],
        "tuning": tuning,
        "roofline": {"bound": "alu", "kernel": "sf32_kernel" if dominant == "sf" else "force32_kernel",
                     "achieved": achieved / 1e12, "peak": peak / 1e12,
                     "unit": "T sin/cos results/s (MUFU)", "frac": achieved / peak, "traffic": traffic,
                     "peak_from": "16 MUFU/clk/SM x 152 SMs x 2070 MHz (derived from the unit count and the "
                                  "maximum SM clock; the probe below measures the per-clock rate on this device)",
                     "probe_per_clk_sm": probe,
                     "other_kernel_frac": (mufu_ops / other) / peak},
        "e2e": {"value": ws * w.N / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(w.N * 3 * 8 + w.N * 8),
                "d2h_bytes_per_step": int(w.N * 3 * 4 + 4 * 8), "steps": e2e_steps,
                "ms_per_call": {"mean": t_e2e * 1e3, "median": float(np.median(t_calls)) * 1e3,
                                "min": float(np.min(t_calls)) * 1e3, "p90": float(np.percentile(t_calls, 90)) * 1e3,
                                "max": float(np.max(t_calls)) * 1e3},
                "timed": "wall clock of rbe2d_sample_k + rbe2d_force(RBE2D_HOST_BUFFERS) on pinned host arrays, "
                         "which returns once the forces and energies are in host memory",
                "l2": "flushed before every call, outside the timed call (as for the device-timed steps)"},
        "gpu_launches": r32["launches"],
        "clocks": r32["clocks"],
    }
    if md_out is not None:
        out["md"] = md_out
    if adjoint_out is not None:
        out["adjoint"] = adjoint_out
    if workloads_out is not None:
        out["workloads"] = workloads_out
    if batch_out is not None:
        out["batched"] = batch_out
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:  # the oracle baseline at N = 1 only
        out["cpu_baseline"] = cpu_baseline(w, p_sample=args.cpu_p)
        out["cpu_baseline"]["workloads"] = oracle_workloads()
    if rank == 0:
        print(json.dumps(out))
    m32.close(); m64.close()
    if ws > 1:
        dist.destroy_process_group()


def _timed_steps(model, N, pos, q, steps, warmup, flush_l2, backward=False):
    """Mean device time (ms) of `steps` steps on the library's stream, L2 flushed before
    each: sample + structure factor + force (or + energy backward)."""
    import torch

    from paper_2405_06333_gb300 import binding as B
    dev = pos.device
    st = torch.cuda.current_stream(dev)
    F = torch.empty((N, 3), dtype=model.out_dtype, device=dev)
    dq = torch.empty(N, dtype=model.out_dtype, device=dev)
    dg = torch.empty(2, dtype=torch.float64, device=dev)
    fl = B.RBE2D_KSPACE | B.RBE2D_IBC

    def step(i):
        B.rbe2d_sample_k(model.ctx, i, None)
        B.rbe2d_structure_factor(model.ctx, N, pos, q, 0, None)
        if backward:
            B.rbe2d_energy_backward(model.ctx, N, pos, q, B.RBE2D_REUSE_SF, 1.0, F, dq, dg)
        else:
            B.rbe2d_force(model.ctx, N, pos, q, fl | B.RBE2D_REUSE_SF, F, None, None)

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    ms = []
    for i in range(steps):
        flush_l2()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        step(warmup + i)
        e1.record(st)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    model.sync_status()
    return float(np.mean(ms))


def adjoint_leg(dev, flush_l2, steps):
    """The energy adjoint (dU/dr, dU/dq, dU/dgamma; rbe2d_energy_backward after the
    structure factor) at the benchmark slab and at the adjoint workload (N = 1e5, P = 300),
    FP32-mixed and FP64 modes: particle-evals/s = N / (sample + structure factor + backward)."""
    import torch

    from paper_2405_06333_gb300 import binding as B
    from paper_2405_06333_gb300.rbe2d import RBE2D
    from paper_2405_06333_gb300.synthetic import WORKLOADS, workload_inputs
    out = {}
    for name in ("slab_n1e6", "adjoint_n1e5"):
        w = WORKLOADS[name]
        ph, qh = workload_inputs(w)
        pos, q = torch.as_tensor(ph, device=dev), torch.as_tensor(qh, device=dev)
        res = {}
        for prec in ("fp32", "fp64"):
            m = RBE2D(w.Lx, w.Ly, w.H, n_max=w.N, P=w.P, gamma_top=w.gamma_top, gamma_bot=w.gamma_bot, M=w.M,
                      Lz=w.Lz, alpha=w.alpha, r_c=w.r_c, seed=w.seed, precision=prec)
            if prec == "fp32":  # the structure factor's and the potential variant's choices, as a user would
                B.rbe2d_sample_k(m.ctx, 0, None)
                scratch = torch.empty((w.N, 3), device=dev)
                tun = B.rbe2d_autotune(m.ctx, w.N, pos, q, B.RBE2D_IBC, scratch)
                tun.update(B.rbe2d_autotune_potential(m.ctx, w.N, pos, q, B.RBE2D_IBC, scratch,
                                                      torch.empty(w.N, device=dev)))
                res["tuning"] = tun
            ms = _timed_steps(m, w.N, pos, q, steps if prec == "fp32" else 3, 2, flush_l2, backward=True)
            m.close()
            res[prec] = {"ms_per_step": ms, "particle_evals_per_s": w.N / (ms * 1e-3)}
        res["speedup_fp32_over_fp64"] = res["fp64"]["ms_per_step"] / res["fp32"]["ms_per_step"]
        res["roofline"] = _step_roofline(8.0 * w.N * w.P, res["fp32"]["ms_per_step"],
                                         "sample + structure factor + backward: 4 sin/cos per (particle, k) pair "
                                         "in each of the two passes")
        out[name] = res
    return out


def _step_roofline(sincos, ms, what):
    """A whole step against the MUFU ceiling: its algorithmic sin/cos results over the
    step time (launch gaps and the small kernels included, so below the kernels' own
    fractions)."""
    peak = MUFU_PER_CLK_SM * SMS * SM_MAX_MHZ * 1e6
    achieved = sincos / (ms * 1e-3)
    return {"bound": "alu", "unit": "sin/cos results/s (MUFU)", "achieved": achieved, "peak": peak,
            "frac": achieved / peak, "work": what, "sincos_per_step": sincos}


def workloads_leg(dev, flush_l2, steps):
    """The metric's step (sample + structure factor + force) at the other workloads, both modes."""
    import torch

    from paper_2405_06333_gb300 import binding as B
    from paper_2405_06333_gb300.rbe2d import RBE2D
    from paper_2405_06333_gb300.synthetic import WORKLOADS, workload_inputs
    out = {}
    for name in ("plain_n1e3", "dielectric_n1e4", "adjoint_n1e5", "thin_n1e6"):
        w = WORKLOADS[name]
        ph, qh = workload_inputs(w)
        pos, q = torch.as_tensor(ph, device=dev), torch.as_tensor(qh, device=dev)
        res = {"N": w.N, "P": w.P, "M": w.M}
        for prec in ("fp32", "fp64"):
            m = RBE2D(w.Lx, w.Ly, w.H, n_max=w.N, P=w.P, gamma_top=w.gamma_top, gamma_bot=w.gamma_bot, M=w.M,
                      Lz=w.Lz, alpha=w.alpha, r_c=w.r_c, seed=w.seed, precision=prec)
            if prec == "fp32":  # launch shapes and FMA-pipe shares for this workload, as a user would
                B.rbe2d_sample_k(m.ctx, 0, None)
                res["tuning"] = B.rbe2d_autotune(m.ctx, w.N, pos, q, B.RBE2D_IBC,
                                                 torch.empty((w.N, 3), device=dev))
            ms = _timed_steps(m, w.N, pos, q, steps if prec == "fp32" else 3, 2, flush_l2)
            m.close()
            res[prec] = {"ms_per_step": ms, "particle_evals_per_s": w.N / (ms * 1e-3)}
        res["speedup_fp32_over_fp64"] = res["fp64"]["ms_per_step"] / res["fp32"]["ms_per_step"]
        out[name] = res
    return out


def batch_leg(dev, steps, tuning=""):
    """512 slabs with N ~ U[200, 20000], Lx = Ly ~ U[10, 60], H ~ U[1, 20], contrasts ~ U[-1, 1],
    P = 200 each: one sampling launch + one persistent launch per step."""
    import torch

    from paper_2405_06333_gb300 import binding as B
    from paper_2405_06333_gb300.synthetic import batched_systems, positions_charges
    systems = batched_systems(n_sys=512, seed=2)
    params, pos, q, off = [], [], [], [0]
    for i, sy in enumerate(systems):
        p_, q_ = positions_charges(sy["N"], sy["Lx"], sy["Ly"], sy["H"], seed=sy["pos_seed"])
        alpha = (sy["N"] / (sy["Lx"] * sy["Ly"] * sy["H"])) ** (1 / 3)
        params.append(B.rbe2d_params(Lx=sy["Lx"], Ly=sy["Ly"], H=sy["H"], Lz=-1, gamma_top=sy["gamma_top"],
                                     gamma_bot=sy["gamma_bot"], M=-1, alpha=alpha, r_c=-1, P=200, seed=100 + i,
                                     eps=1e-4, precision=B.RBE2D_FP32_MIXED, coulomb_k=1.0, real_space=0))
        pos.append(p_); q.append(q_); off.append(off[-1] + sy["N"])
    off = np.array(off, dtype=np.int64)
    b = B.rbe2d_batch_init(params, off, torch.cuda.current_stream(dev))
    P_ = torch.as_tensor(np.concatenate(pos), device=dev)
    Q_ = torch.as_tensor(np.concatenate(q), device=dev)
    F = torch.empty((int(off[-1]), 3), dtype=torch.float32, device=dev)
    if tuning:  # profiler runs: a fixed choice instead of timing under the profiler
        t = [int(x) for x in tuning.split(",")]
        B.rbe2d_batch_set_tuning(b, *t)
        choice = {"sf_chunk": t[0], "f_chunk": t[1], "grid": t[2], "variant": t[3], "set": True}
    else:
        choice = B.rbe2d_batch_autotune(b, P_, Q_, F)
    flags = B.RBE2D_KSPACE | B.RBE2D_IBC
    for i in range(3):
        B.rbe2d_batch_force(b, i, P_, Q_, flags, F)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(steps):
        B.rbe2d_batch_force(b, 10 + i, P_, Q_, flags, F)
    e1.record()
    torch.cuda.synchronize()
    B.rbe2d_batch_sync_status(b)
    ms = e0.elapsed_time(e1) / steps
    B.rbe2d_batch_destroy(b)
    ntot = int(off[-1])
    return {"workload": "512 slabs, N~U[200,20000], Lx=Ly~U[10,60], H~U[1,20], gamma~U[-1,1], P=200 (seed 2)",
            "total_N": ntot, "ms_per_step": ms, "particle_evals_per_s": ntot / (ms * 1e-3),
            "pair_evals_per_s": ntot * 200 / (ms * 1e-3), "launches_per_step": 2, "autotune": choice,
            "roofline": _step_roofline(8.0 * ntot * 200, ms, "sampling launch + persistent launch: 4 sin/cos per "
                                       "(particle, k) pair in each of the two passes"),
            "steps": steps}


def md_leg(w, dev, steps):
    """Langevin MD of the same slab under CUDA-graph replay (one captured step)."""
    import torch

    from paper_2405_06333_gb300 import binding as B
    from paper_2405_06333_gb300.synthetic import lattice_positions_charges
    s = torch.cuda.Stream(dev)
    p = B.rbe2d_params(Lx=w.Lx, Ly=w.Ly, H=w.H, Lz=w.Lz, gamma_top=w.gamma_top, gamma_bot=w.gamma_bot, M=w.M,
                       alpha=w.alpha, r_c=3.0 / w.alpha, P=w.P, seed=w.seed, eps=1e-4,
                       precision=B.RBE2D_FP32_MIXED, coulomb_k=1.0, real_space=1, skin=MD_SKIN)
    ctx = B.rbe2d_init(p, w.N, s)
    pos0, q0 = lattice_positions_charges(w.N, w.Lx, w.Ly, w.H, margin=0.25, seed=1)
    flags = B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_REAL
    # strong damping: the unscreened random start gives large random-batch force noise
    md = B.rbe2d_md_params(dt=5e-4, gamma=10.0, kT=1.0, mass=1.0, sigma_lj=0.5, eps_lj=1.0, sigma_wall=0.25,
                           eps_wall=1.0, noise_seed=3, force_flags=flags)
    with torch.cuda.stream(s):
        pos = torch.as_tensor(pos0, device=dev).contiguous()
        vel = torch.zeros((w.N, 3), dtype=torch.float64, device=dev)
        q = torch.as_tensor(q0, device=dev)
        F = torch.zeros((w.N, 3), dtype=torch.float32, device=dev)
        step = torch.zeros(1, dtype=torch.int64, device=dev)
        stats = torch.zeros(2, dtype=torch.float64, device=dev)
    # the k-space kernels' launch shapes and FMA-pipe shares for this workload (before capture)
    B.rbe2d_sample_k(ctx, 0, None)
    tuning = B.rbe2d_autotune(ctx, w.N, pos, q, B.RBE2D_IBC, F)
    with torch.cuda.stream(s):
        F.zero_()
    s.synchronize()
    t0 = time.perf_counter()
    B.rbe2d_md_step(ctx, w.N, pos, vel, q, F, step, md, B.RBE2D_MD_FORCE, stats)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        B.rbe2d_md_step(ctx, w.N, pos, vel, q, F, step, md, B.RBE2D_MD_STEP, stats)
    # probe: 5 replays; a step slower than 50 ms means something is wrong, stop there
    with torch.cuda.stream(s):
        for _ in range(5):
            g.replay()
    s.synchronize()
    probe_ms = (time.perf_counter() - t0) * 1e3 / 5
    print(f"md probe: {probe_ms:.2f} ms per step (incl. setup)", file=sys.stderr)
    run = 0
    elapsed = 0.0
    if probe_ms < 50.0:
        # chunks of 100 replays on the context's stream; stop if a chunk takes > 5 s
        while run < steps:
            n = min(100, steps - run)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t1 = time.perf_counter()
            with torch.cuda.stream(s):
                e0.record(s)
                for _ in range(n):
                    g.replay()
                e1.record(s)
            s.synchronize()
            elapsed += e0.elapsed_time(e1)
            run += n
            if time.perf_counter() - t1 > 5.0:
                print("md: chunk over 5 s, stopping", file=sys.stderr)
                break
    status = "ok"
    try:
        B.rbe2d_sync_status(ctx)
    except B.RBE2DError as exc:
        status = str(exc)
    ms = elapsed / run if run else probe_ms
    T = 2.0 * float(stats[0]) / (3 * w.N)
    finite = bool(torch.isfinite(pos).all().item())
    # the real-space call (cell list + pair kernel) timed by the library's event timer over
    # eager steps that continue the trajectory, and its roofline
    rs = None
    if run and finite:
        B.rbe2d_timer_enable(ctx, 32, ("real_space", "force", "structure_factor"))
        for _ in range(10):
            B.rbe2d_md_step(ctx, w.N, pos, vel, q, F, step, md, B.RBE2D_MD_STEP, stats)
        kt = B.rbe2d_timer_read(ctx)
        B.rbe2d_timer_enable(ctx, 0)
        rs = real_space_roofline(w, pos.cpu().numpy(), kt["real_space"][0] / max(kt["real_space"][1], 1))
        rs["kernel_ms_per_step"] = {k: v / max(n, 1) for k, (v, n) in kt.items() if n > 0}
    lists = B.rbe2d_md_list_stats(ctx)
    B.rbe2d_destroy(ctx)
    out = {"steps": run, "graph": "one captured BAOAB step, replayed", "ms_per_step": ms,
           "particle_steps_per_s": w.N / (ms * 1e-3), "kinetic_T_end": T, "finite": finite, "status": status,
           "forces": "RBE2D k-space + IBC + erfc real space with images + WCA pairs (sigma 0.5) + WCA walls",
           "real_space": (f"pair lists, skin {MD_SKIN}: {lists['builds']} builds over {run + 16} force evaluations"
                          if lists["enabled"] else "cell scan every step"),
           "dt": 5e-4, "gamma": 10.0, "kT": 1.0, "start": "jittered lattice", "tuning": tuning}
    if rs is not None:
        out["real_space_roofline"] = rs
    return out


def real_space_roofline(w, pos, rs_ms, n_sample=20000):
    """Pairs within r_c that one real-space call evaluates (real and image sources near the
    slab, counted with a k-d tree for a random sample of the charges and scaled to N), and
    the pair rate against the MUFU ceiling: each pair takes three MUFU operations (rsqrt,
    the exponential shared by erfc and the Gaussian term, one reciprocal)."""
    from scipy.spatial import cKDTree
    r_c = 3.0 / w.alpha
    lmax = min(w.M, 2 + int(np.ceil(r_c / w.H))) if (w.M > 0 and (w.gamma_top or w.gamma_bot)) else 0
    z = pos[:, 2]
    src = [pos]
    for l in range(1, lmax + 1):
        sg = -1.0 if l % 2 else 1.0
        for zi in (sg * z + 2.0 * ((l + 1) // 2) * w.H, sg * z - 2.0 * (l // 2) * w.H):
            keep = (zi > -r_c) & (zi < w.H + r_c)
            src.append(np.stack([pos[keep, 0], pos[keep, 1], zi[keep]], axis=1))
    src = np.concatenate(src)
    src[:, 0] = np.mod(src[:, 0], w.Lx)
    src[:, 1] = np.mod(src[:, 1], w.Ly)
    src[:, 2] += r_c
    tree = cKDTree(src, boxsize=[w.Lx, w.Ly, 10.0 * (w.H + 2.0 * r_c)])
    idx = np.random.default_rng(0).choice(len(pos), min(n_sample, len(pos)), replace=False)
    t = pos[idx].copy()
    t[:, 0] = np.mod(t[:, 0], w.Lx)
    t[:, 1] = np.mod(t[:, 1], w.Ly)
    t[:, 2] += r_c
    per = tree.query_ball_point(t, r_c, return_length=True) - 1  # the charge itself is not a pair
    pairs = float(per.mean()) * len(pos)
    peak = MUFU_PER_CLK_SM * SMS * SM_MAX_MHZ * 1e6 / 3.0
    achieved = pairs / (rs_ms * 1e-3)
    return {"kernel": "real-space call", "ms_per_call": rs_ms,
            "pairs_per_call": pairs, "pairs_per_charge": float(per.mean()), "unit": "pairs/s",
            "achieved": achieved, "peak": peak, "frac": achieved / peak, "bound": "alu",
            "peak_from": "16 MUFU/clk/SM x 152 SMs x 2070 MHz / 3 MUFU per pair",
            "sample": f"pairs counted for {len(idx)} random charges of the final configuration with a k-d tree"}


def md_heating(w, dev, steps):
    """Kinetic temperature along eager MD runs of the benchmark slab from the same jittered
    lattice start (dt = 5e-4, gamma = 10, kT = 1): the full force with P = 500, 1000 and
    2000, and without the k-space term (lattice-start relaxation alone).  The random-batch
    force noise has a variance proportional to 1/P (Theorem 2.3); under the Langevin
    thermostat it adds kinetic energy in proportion to it, so the excess T - kT should be
    a constant (the lattice-start transient) plus a term proportional to 1/P.  Reports
    T = 2 KE / 3N over the last half of each run (mean, standard deviation) and the least-
    squares fit T - kT = a + b (500 / P) over the three batch sizes."""
    import torch

    from paper_2405_06333_gb300 import binding as B
    from paper_2405_06333_gb300.synthetic import lattice_positions_charges
    pos0, q0 = lattice_positions_charges(w.N, w.Lx, w.Ly, w.H, margin=0.25, seed=1)
    full = B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_REAL
    runs = {"full_P500": (full, w.P), "full_P1000": (full, 1000), "full_P2000": (full, 2000),
            "no_kspace": (B.RBE2D_IBC | B.RBE2D_REAL, w.P)}
    out = {"steps": steps, "dt": 5e-4, "gamma": 10.0, "kT": 1.0}
    for name, (flags, P) in runs.items():
        s = torch.cuda.Stream(dev)
        p = B.rbe2d_params(Lx=w.Lx, Ly=w.Ly, H=w.H, Lz=w.Lz, gamma_top=w.gamma_top, gamma_bot=w.gamma_bot, M=w.M,
                           alpha=w.alpha, r_c=3.0 / w.alpha, P=P, seed=w.seed, eps=1e-4,
                           precision=B.RBE2D_FP32_MIXED, coulomb_k=1.0, real_space=1, skin=MD_SKIN)
        ctx = B.rbe2d_init(p, w.N, s)
        md = B.rbe2d_md_params(dt=5e-4, gamma=10.0, kT=1.0, mass=1.0, sigma_lj=0.5, eps_lj=1.0, sigma_wall=0.25,
                               eps_wall=1.0, noise_seed=3, force_flags=flags)
        with torch.cuda.stream(s):
            pos = torch.as_tensor(pos0, device=dev).contiguous()
            vel = torch.zeros((w.N, 3), dtype=torch.float64, device=dev)
            q = torch.as_tensor(q0, device=dev)
            F = torch.zeros((w.N, 3), dtype=torch.float32, device=dev)
            step = torch.zeros(1, dtype=torch.int64, device=dev)
            stats = torch.zeros(2, dtype=torch.float64, device=dev)
            ke = torch.zeros(steps, dtype=torch.float64, device=dev)
        B.rbe2d_md_step(ctx, w.N, pos, vel, q, F, step, md, B.RBE2D_MD_FORCE, stats)
        status = "ok"
        t0 = time.perf_counter()
        for i in range(steps):
            B.rbe2d_md_step(ctx, w.N, pos, vel, q, F, step, md, B.RBE2D_MD_STEP, stats)
            with torch.cuda.stream(s):
                ke[i].copy_(stats[0])
            if i % 100 == 99:
                s.synchronize()
                if time.perf_counter() - t0 > 60.0:
                    status = f"stopped after {i + 1} steps (60 s guard)"
                    break
        s.synchronize()
        n = i + 1
        try:
            B.rbe2d_sync_status(ctx)
        except B.RBE2DError as exc:
            status = str(exc)
        B.rbe2d_destroy(ctx)
        T = 2.0 * ke[:n].cpu().numpy() / (3 * w.N)
        half = T[n // 2:]
        out[name] = {"P": P, "flags": "KSPACE|IBC|REAL" if flags & B.RBE2D_KSPACE else "IBC|REAL",
                     "T_last_half_mean": float(half.mean()), "T_last_half_std": float(half.std()),
                     "T_at": {str(k): float(T[k - 1]) for k in (10, 100, 250, 500, 1000, 1500, n) if k <= n},
                     "status": status}
    ps = [500, 1000, 2000]
    ex = [out[f"full_P{p}"]["T_last_half_mean"] - 1.0 for p in ps]
    A = np.stack([np.ones(3), 500.0 / np.array(ps)], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, np.array(ex), rcond=None)
    out["fit_excess_T"] = {"a_transient": float(a), "b_at_P500": float(b),
                           "residuals": [float(e - (a + b * 500.0 / p)) for e, p in zip(ex, ps)]}
    return out


def _oracle_step(w, P_s, step):
    """One bounded oracle evaluation: the full N, the first P_s wave vectors of the batch."""
    import oracle as O
    alpha = w.alpha
    s = O.System(Lx=w.Lx, Ly=w.Ly, H=w.H, Lz=w.Lz, gamma_top=w.gamma_top, gamma_bot=w.gamma_bot, alpha=alpha, M=w.M)
    k = O.sample_k(s, w.seed, step, w.P)[:P_s]
    return s, k


def cpu_baseline(w, p_sample=4, min_seconds=10.0, max_evals=16, p_single=1):
    """The FP64 oracle (OpenMP on the host cores) on the same workload, restricted to
    p_sample of the P wave vectors (at least one per core: the oracle's structure factors
    run one wave vector per thread); evaluations (each with its own k batch) repeat until
    min_seconds of CPU work, and the median time is scaled by P / p_sample.  One more
    evaluation of p_single wave vectors on one thread gives the single-core figure."""
    import oracle as O
    from paper_2405_06333_gb300.synthetic import workload_inputs
    pos, q = workload_inputs(w)
    cores = O.num_threads()
    p_sample = min(w.P, max(p_sample, cores))
    ts = []
    while len(ts) < max_evals and (not ts or sum(ts) < min_seconds):
        s, k = _oracle_step(w, p_sample, len(ts))
        t0 = time.perf_counter()
        O.kspace(s, pos, q, k, O.S(s) / w.P, mode=1)
        ts.append(time.perf_counter() - t0)
    steps = len(ts)
    t_full = float(np.median(ts)) * w.P / p_sample
    O.set_num_threads(1)
    try:
        s, k = _oracle_step(w, p_single, steps)
        t0 = time.perf_counter()
        O.kspace(s, pos, q, k, O.S(s) / w.P, mode=1)
        t1 = time.perf_counter() - t0
    finally:
        O.set_num_threads(cores)
    return {"value": w.N / t_full, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"N={w.N} all particles, {p_sample} of the P={w.P} wave vectors per evaluation "
                      f"(structure factors + forces, re-calibrated FP64 path), median time scaled by "
                      f"P/{p_sample}; {steps} evaluation(s), {np.sum(ts):.1f} s of CPU time",
            "single_core": {"value": w.N / (t1 * w.P / p_single), "unit": UNIT, "cores": 1,
                            "sample": f"{p_single} wave vector(s) on one thread, time scaled by "
                                      f"P/{p_single}; {t1:.1f} s"}}


def oracle_workloads(target_s=2.0):
    """The explicit-image oracle (images built one by one, no recalibration) timed at the
    small configurations, as the random-batch estimator of each workload's batch and as
    the deterministic full k-sum over the Gaussian's box (every k != 0 with |n_d| <= n_d).
    Each timing is a bounded sample of about target_s seconds: a prefix of the batch, or
    wave vectors spread evenly over the full box (unit weights: the cost per wave vector
    does not depend on them), scaled to the whole sum."""
    import oracle as O
    from paper_2405_06333_gb300.synthetic import WORKLOADS, workload_inputs
    out = {}
    for name in ("plain_n1e3", "dielectric_n1e4", "adjoint_n1e5"):
        w = WORKLOADS[name]
        pos, q = workload_inputs(w)
        s = O.System(Lx=w.Lx, Ly=w.Ly, H=w.H, Lz=w.Lz, gamma_top=w.gamma_top, gamma_bot=w.gamma_bot,
                     alpha=w.alpha, M=w.M)
        k = O.sample_k(s, w.seed, 0, w.P)

        def timed(kk, W):
            t0 = time.perf_counter()
            O.kspace(s, pos, q, kk, W, mode=0)
            return time.perf_counter() - t0

        timed(k[:1], 1.0)  # warm-up (thread start)
        t1 = timed(k[:1], 1.0)  # one wave vector: the probe that sizes the samples
        n_rbe = max(1, min(w.P, int(target_s / max(t1, 1e-6))))
        t_rbe = timed(k[:n_rbe], O.S(s) / w.P) * w.P / n_rbe
        nd = [O.nmax(w.alpha, L) for L in (w.Lx, w.Ly, w.Lz)]
        side = [2 * n + 1 for n in nd]
        K = int(np.prod(side)) - 1
        n_full = max(1, min(K, int(target_s / max(t1, 1e-6))))
        flat = np.linspace(0, K - 1, n_full).astype(np.int64)
        flat = flat + (flat >= K // 2)  # skip the centre (k = 0)
        kf = np.stack(np.unravel_index(flat, side), axis=1).astype(np.int32) - np.asarray(nd, dtype=np.int32)
        t_full = timed(kf, 1.0) * K / n_full
        out[name] = {"N": w.N, "P": w.P, "M": w.M, "cores": O.num_threads(),
                     "explicit_rbe": {"ms_per_eval": t_rbe * 1e3, "particle_evals_per_s": w.N / t_rbe,
                                      "sample": f"{n_rbe} of the P={w.P} wave vectors, scaled by P/{n_rbe}"},
                     "full_k_sum": {"ms_per_eval": t_full * 1e3, "particle_evals_per_s": w.N / t_full,
                                    "wave_vectors": K,
                                    "sample": f"{n_full} of the {K} wave vectors, scaled by {K}/{n_full}"}}
    return out


def _reference_sample(N, P, cores, cpu_p, rate, steps, warmup):
    """(particles, wave vectors) of one reference step: at least one wave vector per core,
    and a prefix of the particles sized from the measured pair rate so that the run's
    steps take about two minutes in all, at most 2 s each."""
    p_s = min(P, max(cpu_p, cores))
    budget = min(2.0, 120.0 / max(1, steps + min(warmup, 1)))
    pairs = max(1000.0, rate * budget)
    n_s = int(max(2, min(N, pairs // p_s))) & ~1
    return n_s, p_s


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2405_06333_gb300.synthetic import WORKLOADS
    w = WORKLOADS[args.workload]
    import oracle as O
    from paper_2405_06333_gb300.synthetic import workload_inputs
    # all the host cores this process may use (torch.distributed.run sets OMP_NUM_THREADS=1)
    O.set_num_threads(len(os.sched_getaffinity(0)))
    pos, q = workload_inputs(w)
    # the pair rate of the oracle on this host, from one wave vector over a prefix of the
    # particles; then each step's sample (a prefix of N_s particles against P_s wave
    # vectors) is sized so that the whole --steps/--warmup run takes about two minutes
    # (the oracle's structure factors run one wave vector per thread and its forces one
    # particle per thread, so a sample holds at least as many wave vectors as cores)
    cores = O.num_threads()
    p_min = min(w.P, max(args.cpu_p, cores))
    n_cal = min(w.N, 20000)
    s, k = _oracle_step(w, p_min, 0)
    O.kspace(s, pos[:n_cal], q[:n_cal], k, O.S(s) / w.P, mode=1)  # thread start
    t0 = time.perf_counter()
    O.kspace(s, pos[:n_cal], q[:n_cal], k, O.S(s) / w.P, mode=1)
    rate = n_cal * p_min / max(time.perf_counter() - t0, 1e-9)  # (particle, wave vector) pairs per second
    N_s, P_s = _reference_sample(w.N, w.P, cores, args.cpu_p, rate, args.steps, args.warmup)
    for i in range(min(args.warmup, 1)):
        s, k = _oracle_step(w, P_s, i)
        O.kspace(s, pos[:N_s], q[:N_s], k, O.S(s) / w.P, mode=1)
    ts = []
    for i in range(args.steps):
        s, k = _oracle_step(w, P_s, args.warmup + i)
        t0 = time.perf_counter()
        O.kspace(s, pos[:N_s], q[:N_s], k, O.S(s) / w.P, mode=1)
        ts.append(time.perf_counter() - t0)
    t_step = float(np.mean(ts))
    # one step is a bounded sample: N_s particles against P_s of the P wave vectors, i.e.
    # N_s P_s / P particle-evals of the full workload
    value = N_s * (P_s / w.P) / t_step
    sample = (f"each step: the first {N_s} of the N={w.N} particles against {P_s} of the P={w.P} wave vectors "
              f"(structure factors + forces, re-calibrated FP64 oracle) = {N_s}*{P_s}/{w.P} particle-evals of "
              f"the workload; sized for about 2 minutes over {args.steps} steps")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": _workload_config(w, ws),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-p", type=int, default=4, help="wave vectors per oracle evaluation")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="FP32 path only (for profiler runs)")
    ap.add_argument("--no-md", action="store_true", help="skip the MD leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched leg")
    ap.add_argument("--md-steps", type=int, default=1000)
    ap.add_argument("--md-only", action="store_true", help="only the MD leg (for profiler runs)")
    ap.add_argument("--no-extra", action="store_true", help="skip the adjoint and other-workload legs")
    ap.add_argument("--batch-only", action="store_true", help="only the batched leg (for profiler runs)")
    ap.add_argument("--adjoint-only", action="store_true", help="only the adjoint leg (for profiler runs)")
    ap.add_argument("--tuning", default="", help="sf_poly,force_poly,sf_shape,force_shape instead of the autotuner")
    ap.add_argument("--batch-steps", type=int, default=50)
    ap.add_argument("--batch-tuning", default="",
                    help="sf_chunk,f_chunk,grid,variant for the batched leg instead of its autotuner")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
