#!/usr/bin/env python
"""Benchmark of the fast-hybrid 2D scattering path on GB300.

One step = the whole path over one synthetic problem:
  a1 nodes/tables -> a2 CFIE assembly -> a3 LU + solve (every omega_j > 0)
  -> a4 window spectra -> a5 target fields -> a6 synthesis weights
  -> a7 synthesis contraction.

Headline workload (`--workload kite_wide`, the wide-band precision
configuration): kite obstacle, 40-pulse incident train over [0, 400], 512
frequencies on [0, 160] (511 solves), N_j by 8 points per wavelength
(64..1920), 1024 targets on r = 3, 4096 times up to T = 1e4.  `value` is
frequency solves/s of whole steps with inputs resident in HBM in the
mixed precision (`--precision`, default BF16 tensor-core LU + FP64-class
refinement); `e2e` the same through the host-pointer C-ABI calls with the
host<->device copies inside the timed region.  Beside it, in the same run:

* the plain FP64 GPU path on the same workload (fewer steps), its solves/s
  and the mixed/FP64 ratio; the TF32 tensor-core LU on the same workload;
* the measured error of the timed output: u against the FP64 GPU u at all
  targets and times, densities and target fields against the FP64 oracle at
  sampled frequencies;
* the 256-frequency kite (N 64..480) in both precisions, with u against the
  oracle's full run at all 1024 targets x 4096 times;
* the batching configuration (32 star obstacles x 128 frequencies, N up to
  ~900, one batched context);
* peaks measured on this GPU (FP64 / FP32 FMA chains, TF32 / BF16 tcgen05
  MMAs), every phase against its roofline, the oracle on the host cores.

L2 is flushed (256 MiB write) between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--precision fp64|mixed|tf32|bf16] [--workload kite_wide|kite_pulses]
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fh_inputs as fi  # noqa: E402

METRIC = "frequency solves/s & time samples/s at 1e-10 rel err (mixed vs FP64); p50/p99"
# arithmetic each --precision computes in
DTYPES = {"fp64": "f64",
          "mixed": "f64 + f32 (LU) + f32-pair (Hankel, synthesis)",
          "tf32": "f64 + tf32x3 tensor (LU) + f32-pair (Hankel, synthesis)",
          "bf16": "f64 + bf16x3 tensor (LU) + f32-pair (Hankel, synthesis)"}
WORKLOADS = {
    "kite_wide": (lambda: fi.kite_wide(),
                  "kite_wide: kite, 40 pulses over [0,400], J=512 on [0,160], N=64..1920 (8 ppw), "
                  "1024 targets, 4096 times to T=1e4"),
    "kite_pulses": (lambda: fi.kite_pulses(),
                    "kite_pulses: kite, 40 pulses over [0,400], J=256 on [0,40], N=64..480 (8 ppw), "
                    "1024 targets, 4096 times to T=1e4"),
}
# frequencies at which densities / target fields of the wide-band workload are
# checked against the oracle (its 511 solves take minutes on the host)
WIDE_CHECK_J = [1, 40, 128, 255, 384, 470, 511]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp64", "mixed", "tf32", "bf16"])
    ap.add_argument("--workload", default="kite_wide", choices=list(WORKLOADS))
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the FP64 leg on the headline workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline leg only (no FP64 leg, other workloads or oracle accuracy)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default schedule instead of running the autotuner at set-up")
    ap.add_argument("--tuning", default=None,
                    help="schedule given explicitly instead of autotuned, e.g. "
                         "assemble_group=8,field_group=4,field_chunk=64,lu_rows_per_cta=512,lu_early=20")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------- algorithmic work

def lu_flops(N):
    """Complex LU with partial pivoting: (8/3) N^3 real flops per system."""
    N = np.asarray(N, dtype=np.float64)
    return float(np.sum(8.0 / 3.0 * N ** 3))


def contract_flops(n_x, n_T, J):
    """u = [Vr|Vi][Gr;Gm]: 2 flops per multiply-add over inner dimension 2J."""
    return 2.0 * n_x * n_T * 2 * J


def window_pairs(wl):
    """(time, window) pairs of the synthesis weights per step."""
    span = wl.t0 + wl.dt * (wl.a.size - 1)
    K = 0
    while 1.5 * wl.H * K - wl.H < span:
        K += 1
    return wl.T.size * max(K, 1)


# Pipe utilisation of the ALU-bound kernels (the hardware-anchored fraction of
# their roofline), from ncu captures of one launch of each kernel on the
# wide-band kite (summaries in profiles/).  Their algorithmic rates are given
# in the method's own units (matrix entries/s, target-node pairs/s).
NCU_PIPE = {"lu_factor_tc_kernel": {"tensor_pipe_active_pct": 9.8, "issue_active_pct": 17.9,
                                    "dram_throughput_pct": 8.9,
                                    "capture": "profiles/lu_factor_tc_kite_wide.md (BF16)"}}
# DRAM bytes (read + write) of the dominant kernels per step, from the same
# captures (None where no capture of the current kernel exists): the LU's
# capture of the clusters of 4 CTAs of the reduced case (13 systems, N
# 1568..1920: 5.44 GB), scaled to the headline workload's factorisation by
# sum N^3 (13.3x).
MEASURED_TRAFFIC = {"lu_factor_tc_kernel": 7.24e10}


def phase_rooflines(wl, precision, ms, iters, peaks, contract_tc=False):
    """Achieved against peak per phase: the method's work per step over the
    phase time.  Tensor-core phases: flops of the method (not of the split
    operands) against the measured tcgen05 rate of their operand type; the
    refinement: bytes against the measured copy bandwidth; ALU phases: their
    own units per second, the fraction from ncu pipe utilisation."""
    N = wl.N[1:].astype(np.float64)
    mixed = precision != "fp64"
    out = {}

    def put(phase, kernel, bound, work, unit, peak=None, peak_src=None, scale=1.0, extra=None):
        if ms.get(phase, 0) <= 0:
            return
        ach = work / (ms[phase] * 1e-3) / scale
        d = {"kernel": kernel, "bound": bound, "unit": unit, "work_per_step": work, "achieved": ach,
             "ms_per_step": ms[phase]}
        if peak:
            d.update(peak=peak, frac=ach / peak, peak_source=peak_src)
        if kernel in NCU_PIPE and precision == "bf16":
            d["ncu"] = NCU_PIPE[kernel]
        if extra:
            d.update(extra)
        out[phase] = d

    put("assemble", "assemble_group_df_kernel" if mixed else "assemble_group_kernel", "alu",
        float(np.sum(N * N)), "entries/s")
    if precision == "fp64":
        put("factor", "lu_solve_fp64_kernel", "alu", lu_flops(N), "TFLOP/s", peaks.get("fp64_tflops"),
            "measured FP64 FMA-chain rate of this GPU (fh_probe_fma_peak)", 1e12)
    elif precision == "mixed":
        put("factor", "lu_factor_fp32_kernel", "alu", lu_flops(N), "TFLOP/s", peaks.get("fp32_tflops"),
            "measured FP32 FMA-chain rate of this GPU (fh_probe_fma_peak)", 1e12)
    else:
        key = "tf32_tflops" if precision == "tf32" else "bf16_tflops"
        put("factor", "lu_factor_tc_kernel", "tensor", lu_flops(N), "TFLOP/s", peaks.get(key),
            f"measured dense {precision.upper()} tcgen05 MMA rate of this GPU (fh_probe_mma_peak, burst); "
            "work (8/3) sum N^3 of the method (the 3-term operand split is not counted)", 1e12)
    if mixed:
        put("refine", "refine_resid_kernel", "hbm", 24.0 * float(np.sum(N * N)) * max(iters, 1), "GB/s",
            peaks.get("hbm_gbs"), "measured copy bandwidth (MEASURED_PEAKS.json); bytes: the "
            "double-float matrix (16 B/entry, residual) and the FP32 factors (8 B/entry, solves) "
            "per sweep x the largest sweep count", 1e9)
    put("field", "field_partial_df_kernel" if mixed else "field_partial_kernel", "alu",
        float(wl.n_x) * float(np.sum(N)), "pairs/s")
    put("weights", "weights_kernel", "alu", float(window_pairs(wl)), "(t,k) pairs/s",
        extra={"frequencies": wl.J})
    cf = contract_flops(wl.n_x, wl.T.size, wl.J)
    if contract_tc:
        put("contract", "contract_tc_kernel", "tensor", cf, "TFLOP/s", peaks.get("bf16_tflops"),
            "measured dense BF16 tcgen05 MMA rate (fh_probe_mma_peak); work 2 n_x n_T (2J) of the "
            "method (the 36 exact slice-pair products are not counted)", 1e12)
    elif mixed:
        put("contract", "contract_df_kernel", "alu", cf, "TFLOP/s",
            peaks.get("fp32_tflops") and peaks["fp32_tflops"] / 11.0,
            "measured FP32 FMA rate / 11 FP32 instructions per double-float multiply-add", 1e12)
    else:
        put("contract", "contract_kernel", "alu", cf, "TFLOP/s", peaks.get("fp64_tflops"),
            "measured FP64 FMA-chain rate (fh_probe_fma_peak)", 1e12)
    return out


def measure_peaks(F, device):
    peaks = {}
    try:
        mp_ = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peaks["hbm_gbs"] = mp_.get("hbm_gbs")
        peaks["bf16_cublas_tflops"] = mp_.get("bf16_tflops")
        peaks["bf16_cublas_tflops_sustained"] = mp_.get("bf16_tflops_sustained")
    except Exception:
        peaks["hbm_gbs"] = None
    peaks["fp64_tflops"] = F.fh_probe_fma_peak(device, True, 4096)
    peaks["fp32_tflops"] = F.fh_probe_fma_peak(device, False, 8192)
    peaks["tf32_tflops"] = F.fh_probe_mma_peak(device, 2, 20000)
    peaks["bf16_tflops"] = F.fh_probe_mma_peak(device, 1, 20000)
    peaks["source"] = ("fp64/fp32: independent FMA chains on every SM; tf32/bf16: back-to-back "
                       "tcgen05 MMAs (128x256, one K step) from shared memory, one CTA per SM; "
                       "hbm: MEASURED_PEAKS.json copy bandwidth")
    return peaks


# ------------------------------------------------------------ CPU oracle

def _oracle_jobs(out_path, jobs):
    """Oracle work for the benchmark, run in a process of its own (spawned
    before the parent touches the GPU) while the GPU legs run.  Writes an .npz
    of results and timings."""
    sys.path.insert(0, ROOT)
    try:    # leave the first two cores to the process driving the GPU
        cores = sorted(os.sched_getaffinity(0))
        if len(cores) > 4:
            os.sched_setaffinity(0, cores[2:])
    except (AttributeError, OSError):
        pass
    import oracle as O
    res = {}
    if "kite_pulses_full" in jobs:
        wl = fi.kite_pulses()
        t0 = time.perf_counter()
        psi = O.solve_all(wl)
        t_solve = time.perf_counter() - t0
        t1 = time.perf_counter()
        s, B = O.window_spectra(wl.a, wl.t0, wl.dt, wl.H, wl.omega)
        V = O.target_fields(wl, psi)
        u = O.synthesize(B, s, wl.omega, V, wl.T)
        res["kp_u"] = u
        res["kp_t_solve"] = t_solve
        res["kp_t_step"] = time.perf_counter() - t0
        res["kp_t_time_side"] = time.perf_counter() - t1
    if "kite_wide_sampled" in jobs:
        wl = fi.kite_wide()
        xs = wl.x.reshape(-1, 2)[::64].reshape(-1)           # 16 targets
        ts, Ns, psis, Vs = [], [], [], []
        for j in WIDE_CHECK_J:
            t0 = time.perf_counter()
            psi = O.solve_density(wl.curve, int(wl.N[j]) // 2, float(wl.omega[j]), wl.c, wl.p)
            ts.append(time.perf_counter() - t0)
            Ns.append(int(wl.N[j]))
            psis.append(psi)
            Vs.append(O.target_field(wl.curve, int(wl.N[j]) // 2, float(wl.omega[j]), psi, xs, wl.c))
        res["kw_j"] = np.asarray(WIDE_CHECK_J)
        res["kw_t"] = np.asarray(ts)
        res["kw_N"] = np.asarray(Ns)
        res["kw_psi"] = np.concatenate(psis)
        res["kw_V"] = np.stack(Vs, 1)
        # time side of the step on a sample: spectra in full, synthesis for 16 targets
        rng = np.random.default_rng(0)
        t0 = time.perf_counter()
        s, B = O.window_spectra(wl.a, wl.t0, wl.dt, wl.H, wl.omega)
        Vr = rng.standard_normal((16, wl.J)) + 1j * rng.standard_normal((16, wl.J))
        O.synthesize(B, s, wl.omega, Vr, wl.T)
        res["kw_t_synth16"] = time.perf_counter() - t0
    np.savez(out_path, **res)


def start_oracle(jobs):
    """Spawn the oracle process (before any CUDA call in this process).  It
    runs on all host cores but the first two (BLAS threads set to match), so
    that the thread launching the GPU work is not starved."""
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    n = max(1, cpu_cores() - 2) if cpu_cores() > 4 else cpu_cores()
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ.update(OMP_NUM_THREADS=str(n), OPENBLAS_NUM_THREADS=str(n))
    ctx = mp.get_context("spawn")
    p = ctx.Process(target=_oracle_jobs, args=(path, jobs), daemon=True)
    p.start()
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    return p, path, n


def finish_oracle(p, path, threads, timeout=900):
    p.join(timeout)
    if p.is_alive():
        p.terminate()
        return None
    try:
        d = dict(np.load(path))
        d["threads"] = threads
    except Exception:
        d = None
    try:
        os.unlink(path)
    except OSError:
        pass
    return d


def n3_fit(N, t):
    """Non-negative least squares t = c0 + c2 N^2 + c3 N^3 over the sampled
    solves (assembly ~ N^2, LU ~ N^3, a fixed per-solve cost); returns
    (c0, c2, c3)."""
    from scipy.optimize import nnls
    N = np.asarray(N, dtype=float)
    A = np.stack([np.ones_like(N), N ** 2, N ** 3], 1)
    sc = A.max(axis=0)
    c, _ = nnls(A / sc, np.asarray(t, dtype=float))
    return c / sc


def oracle_solve_sample(wl, stride, offset):
    """The oracle's frequency solves (assembly + LU + solve) for every
    stride-th frequency of the workload, so that the sample has the
    workload's mix of N.  Returns (solves, seconds, N list, per-solve s)."""
    import oracle as O
    js = list(range(1 + offset, wl.J, stride))
    ts = []
    for j in js:
        t0 = time.perf_counter()
        O.solve_density(wl.curve, int(wl.N[j]) // 2, float(wl.omega[j]), wl.c, wl.p)
        ts.append(time.perf_counter() - t0)
    return len(js), float(sum(ts)), [int(wl.N[j]) for j in js], ts


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """Max of a per-rank scalar over all ranks (identity at world size 1)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- arms

def run_reference(args, world, rank):
    """The oracle as it stands on the host cores.  Each step is a bounded
    sample of the workload: the frequency solves of every 64th frequency
    (eight solves spanning the workload's N range, assembly + LU + solve);
    value = solves done / time taken.  Warm-up steps solve one frequency."""
    if rank != 0:
        return
    wl = WORKLOADS[args.workload][0]()
    stride = 64 if wl.J > 300 else 32
    for w in range(args.warmup):
        oracle_solve_sample(wl, wl.J, w % 2)
    n_tot, t_tot, Ns = 0, 0.0, []
    for k in range(args.steps):
        n, t, N, _ = oracle_solve_sample(wl, stride, (7 * k) % stride)
        n_tot += n
        t_tot += t
        Ns += N
    value = n_tot / t_tot
    desc = (f"oracle (numpy/scipy FP64, {cpu_cores()} host cores) frequency solves of every "
            f"{stride}th frequency per step (offset rotating by 7), N in [{min(Ns)}, {max(Ns)}]; "
            f"{n_tot} solves in {t_tot:.1f} s; fields and synthesis not included")
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOADS[args.workload][1], "precision": "fp64",
                   "step": f"bounded sample: every {stride}th frequency's solve"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


class Leg:
    """One context driven through the whole path on one workload: set-up
    (schedule autotuning, untimed), device-resident timed steps, a kernel
    timing pass and the end-to-end host-pointer steps."""

    def __init__(self, F, torch, local, stream, wl, precision, args, autotune=True):
        self.F, self.torch, self.wl = F, torch, wl
        self.prec_name = precision
        prec = {"fp64": F.FH_FP64, "mixed": F.FH_MIXED_FP32, "tf32": F.FH_MIXED_TF32,
                "bf16": F.FH_MIXED_BF16}[precision]
        self.pr = F.Problem(local, prec)
        self.stream = stream
        F.fh_set_stream(self.pr.ctx, stream.cuda_stream)
        dev = torch.device("cuda", local)
        self.d_a = torch.tensor(wl.a, device=dev, dtype=torch.float64)
        self.d_x = torch.tensor(wl.x, device=dev, dtype=torch.float64)
        self.d_T = torch.tensor(wl.T, device=dev, dtype=torch.float64)
        self.d_u = torch.empty(wl.n_x * wl.T.size, device=dev, dtype=torch.float64)
        torch.cuda.synchronize()
        self.tuning = {"autotuned": False, "setting": F.fh_get_tuning(self.pr.ctx)}
        if args.tuning:
            F.fh_set_tuning(self.pr.ctx, **{k: int(v) for k, v in
                                            (kv.split("=") for kv in args.tuning.split(","))})
            self.tuning = {"autotuned": False, "setting": F.fh_get_tuning(self.pr.ctx)}
        elif autotune and not args.no_tune:
            F.fh_discretize(self.pr.ctx, wl.curve, wl.omega, wl.N, wl.c, wl.p)
            t0 = time.perf_counter()
            chosen, best_ms = F.fh_autotune(self.pr.ctx, wl.x, reps=3)
            self.tuning = {"autotuned": True, "setting": chosen, "best_ms": best_ms,
                           "tune_s": time.perf_counter() - t0}
        self.stats = {}

    def step(self):
        F, wl, ctx = self.F, self.wl, self.pr.ctx
        F.fh_discretize(ctx, wl.curve, wl.omega, wl.N, wl.c, wl.p)
        st = F.fh_solve_frequencies(ctx)
        self.stats["iters"] = st.refine_iters_max
        self.stats["resid"] = st.residual_max
        F.fh_window_spectra_dev(ctx, self.d_a, wl.t0, wl.dt, wl.H)
        F.fh_sample_dev(ctx, self.d_x, self.d_T, self.d_u)

    def timed(self, steps, warmup, flush, clocks=None, barrier=lambda: None):
        torch = self.torch
        for _ in range(max(warmup, 0)):
            self.step()
        torch.cuda.synchronize()
        self.F.fh_get_timings(self.pr.ctx, reset=True)
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        ev = []
        for k in range(steps):
            flush.fill_(float(k))                      # L2 flush between steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            self.step()
            e1.record(self.stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop() if clocks else None
        per_step = [a.elapsed_time(b) for a, b in ev]
        tim = self.F.fh_get_timings(self.pr.ctx, reset=True)
        launches = sum(v["launches"] for v in tim.values())
        return per_step, launches, clk

    def phases(self, reps, flush):
        F = self.F
        F.fh_set_timing(self.pr.ctx, True)
        for k in range(reps):
            flush.fill_(float(k))
            self.step()
        ph = F.fh_get_timings(self.pr.ctx, reset=True)
        F.fh_set_timing(self.pr.ctx, False)
        return {n: v["ms"] / reps for n, v in ph.items()}

    def e2e(self, steps, flush):
        F, wl, torch = self.F, self.wl, self.torch

        def pinned(arr):
            return torch.from_numpy(np.ascontiguousarray(arr)).pin_memory().numpy()
        a_p, x_p, T_p, om_p = pinned(wl.a), pinned(wl.x), pinned(wl.T), pinned(wl.omega)
        u_host = torch.empty(wl.n_x * wl.T.size, dtype=torch.float64).pin_memory().numpy()
        times = []
        for k in range(steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            F.fh_discretize(self.pr.ctx, wl.curve, om_p, wl.N, wl.c, wl.p)
            F.fh_solve_frequencies(self.pr.ctx)
            F.fh_window_spectra(self.pr.ctx, a_p, wl.t0, wl.dt, wl.H)
            F.fh_sample(self.pr.ctx, x_p, T_p, out=u_host)
            times.append(time.perf_counter() - t0)
        assert np.all(np.isfinite(u_host))
        h2d = wl.a.nbytes + wl.x.nbytes + wl.T.nbytes + wl.omega.nbytes + wl.N.nbytes
        return times, int(h2d), int(u_host.nbytes)

    def resample_timed(self, steps, flush):
        """Time samples on the resident target fields (no fresh step F5):
        fh_resample_p_dev at the workload's times, per call ms."""
        torch = self.torch
        ev = []
        for k in range(steps):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            self.F.fh_resample_p_dev(self.pr.ctx, 0, self.d_T, self.d_u)
            e1.record(self.stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    def u(self):
        self.stream.synchronize()
        return self.d_u.cpu().numpy().reshape(self.wl.n_x, self.wl.T.size)

    def density(self, j):
        return self.F.fh_get_density(self.pr.ctx, int(j), int(self.wl.N[j]))

    def target_field(self):
        return self.F.fh_get_target_field(self.pr.ctx, self.wl.n_x, self.wl.J)

    def close(self):
        self.pr.close()


def summary(per_step, units):
    total = sum(per_step)
    return {"value": units * len(per_step) / (total / 1e3), "ms_per_step": total / len(per_step),
            "p50_ms": float(np.percentile(per_step, 50)), "p99_ms": float(np.percentile(per_step, 99)),
            "steps": len(per_step)}


PRECISIONS = None   # name -> fh precision code, filled once the binding is loaded


def batch_leg(F, torch, local, stream, flush, steps, warmup, precision):
    """32 star obstacles x 128 frequencies on [0, w_max], w_max ~ U(20, 100),
    N by 8 points per wavelength (64 .. ~900), all in one batched context
    (one launch per kernel for all problems), in the bench's precision; 256
    targets x 512 times per problem.  solves/s of whole batched steps."""
    probs = fi.star_batch()
    sig = fi.pulse_train(3, n=8, span=80.0, fmin=4.0, fmax=16.0)
    t0s, dt = -10.0, 0.01
    a = fi.sample_signal(sig, t0s, dt, int(np.ceil((sig.t_end - t0s) / dt)) + 1)
    dev = torch.device("cuda", local)
    x = fi.targets_on_circle(256, 3.0)
    T = np.sort(np.random.default_rng(4).uniform(0.0, 1e4, 512))
    d_a = torch.tensor(a, device=dev, dtype=torch.float64)
    d_x = torch.tensor(x, device=dev, dtype=torch.float64)
    d_T = torch.tensor(T, device=dev, dtype=torch.float64)
    d_u = torch.empty(x.size // 2 * T.size, device=dev, dtype=torch.float64)
    torch.cuda.synchronize()
    ctx = F.fh_create(local, PRECISIONS[precision])
    F.fh_set_stream(ctx, stream.cuda_stream)
    curves, oms, Ns = [p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs]
    F.fh_discretize_batch(ctx, curves, oms, Ns)
    tuning, _ = F.fh_autotune(ctx, x, reps=2)
    S = sum(len(o) - 1 for o in oms)

    def step():
        F.fh_discretize_batch(ctx, curves, oms, Ns)
        F.fh_solve_frequencies(ctx)
        for q in range(len(probs)):
            F.fh_window_spectra_p_dev(ctx, q, d_a, t0s, dt)
            F.fh_sample_p_dev(ctx, q, d_x, d_T, d_u)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev = []
    for k in range(steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    per = [p.elapsed_time(q) for p, q in ev]
    F.fh_destroy(ctx)
    out = summary(per, S)
    Nall = np.concatenate([n[1:] for n in Ns])
    out.update({"workload": "star_batch: 32 stars r=1+sum_{k<=5} a_k cos(kt+phi_k), a~U(0,0.1), "
                            "128 freqs each on [0,w_max], w_max~U(20,100), N 8 ppw "
                            f"({int(Nall.min())}..{int(Nall.max())}); 256 targets x 512 times per problem",
                "precision": precision, "solves_per_step": S, "tuning": tuning,
                "time_samples_per_s": len(probs) * x.size // 2 * T.size * len(per) / (sum(per) / 1e3)})
    return out


def split_synthesis_leg(F, torch, local, stream, steps, precision):
    """The 2D synthesis with the low-frequency split (FCC on (0, w_c], FC(Gram)
    on [w_c, W]) on the 256-frequency kite: densities and target fields of
    the mesh and of the 24 singular frequencies from the solver, then
    fh_synthesize_sing for 1024 targets x 4096 times, timed with CUDA events."""
    wl = fi.kite_pulses()
    j_c = 5
    dev = torch.device("cuda", local)
    pr = F.Problem(local, PRECISIONS[precision])
    F.fh_set_stream(pr.ctx, stream.cuda_stream)
    pr.discretize(wl.curve, wl.omega, wl.N, wl.c, wl.p)
    pr.solve()
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    pr.sample(wl.x, wl.T[:2])
    V = F.fh_get_target_field(pr.ctx, wl.n_x, wl.J)
    s, B = F.fh_get_window_spectra(pr.ctx, wl.J)
    pr.close()
    osg = F.fh_sing_frequencies(wl.omega[j_c])
    ctx = F.fh_create(local, PRECISIONS[precision])
    P = osg.size
    F.fh_discretize_batch(ctx, [wl.curve] * P, [np.array([0.0, w]) for w in osg],
                          [np.array([64, 64], dtype=np.int32)] * P, ps=[wl.p] * P)
    F.fh_solve_frequencies(ctx)
    Vs = np.empty((wl.n_x, P), dtype=np.complex128)
    Bs = np.empty((B.shape[0], P), dtype=np.complex128)
    for q in range(P):
        F.fh_window_spectra_p(ctx, q, wl.a, wl.t0, wl.dt, wl.H)
        F.fh_sample_p(ctx, q, wl.x, wl.T[:2])
        Vs[:, q] = F.fh_get_target_field(ctx, wl.n_x, 2)[:, 1]
        Bs[:, q] = F.fh_get_window_spectra_p(ctx, q, 2)[1][:, 1]
    F.fh_destroy(ctx)

    def d(a):
        a = np.ascontiguousarray(a)
        return torch.tensor((a.view(np.float64) if np.iscomplexobj(a) else a).ravel(), device=dev)
    d_s, d_B, d_Bs = d(s), d(B), d(Bs)
    d_V, d_Vs, d_T = d(V.T), d(Vs.T), d(wl.T)
    d_u = torch.empty(wl.n_x * wl.T.size, device=dev, dtype=torch.float64)
    torch.cuda.synchronize()
    F.fh_synthesize_sing(wl.J, float(wl.omega[-1]), j_c, d_s, d_B, d_Bs, d_V, d_Vs, d_T, d_u,
                         stream.cuda_stream)
    ev = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        F.fh_synthesize_sing(wl.J, float(wl.omega[-1]), j_c, d_s, d_B, d_Bs, d_V, d_Vs, d_T, d_u,
                             stream.cuda_stream)
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    per = [a.elapsed_time(b) for a, b in ev]
    ms = sum(per) / len(per)
    assert bool(torch.isfinite(d_u).all())
    return {"workload": WORKLOADS["kite_pulses"][1] + f"; w_c = omega_{j_c}, 24 singular frequencies",
            "ms_per_call": ms, "time_samples_per_s": wl.n_x * wl.T.size / (ms * 1e-3),
            "calls": len(per), "extra_solves": P}


def serving_leg(rates, n_requests, precision):
    """Continuous-batching server at the serving configuration's shape (star
    obstacles, 128 frequencies on [0, w_max], w_max ~ U(10, 120), pulse or
    chirp signals, 256-4096 targets and 1-100 queries of 16 times in [0, 1e4]
    per request), Poisson arrivals, in the bench's precision: p50/p99 request
    latency and throughput per arrival rate."""
    from paper_1807_02718_gb300 import serve as SV
    out = []
    for i, rate in enumerate(rates):
        st = SV.run_stream(rate, n_requests, seed=11 + i, precision=PRECISIONS[precision])
        out.append(st)
    return out


def run_gpu(args, world, rank, local):
    extra = not args.no_extra and world == 1 and rank == 0
    oracle_proc = None
    if extra:
        # the oracle runs in a spawned process beside the GPU legs
        oracle_proc = start_oracle(["kite_pulses_full", "kite_wide_sampled"]
                                   if args.workload == "kite_wide" else ["kite_pulses_full"])
    import torch
    import torch.distributed as dist
    from paper_1807_02718_gb300 import build
    from paper_1807_02718_gb300 import fh as F

    build.build()
    global PRECISIONS
    PRECISIONS = {"fp64": F.FH_FP64, "mixed": F.FH_MIXED_FP32, "tf32": F.FH_MIXED_TF32, "bf16": F.FH_MIXED_BF16}
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # One explicit stream for the library, the L2 flush and the timing events
    # (torch's default stream has the NULL handle, which would leave the
    # library on its own stream, unordered with the events).
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 8, device=dev, dtype=torch.float64)
    peaks = measure_peaks(F, local)

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- headline: mixed precision on the headline workload ----
    wl = WORKLOADS[args.workload][0]()
    S = wl.J - 1
    n_x, n_T = wl.n_x, wl.T.size
    leg = Leg(F, torch, local, stream, wl, args.precision, args)
    clocks = ClockSampler(local)
    per_step, launches, clk = leg.timed(args.steps, args.warmup, flush, clocks, barrier)
    total_ms = max_over_ranks(sum(per_step), world, dev)
    value = world * S * args.steps / (total_ms / 1e3)
    samples_per_s = world * n_x * n_T * args.steps / (total_ms / 1e3)
    u_mixed = leg.u()
    res = leg.resample_timed(max(3, args.steps // 2), flush)
    resident = {"ms_per_call": sum(res) / len(res),
                "time_samples_per_s": n_x * n_T * len(res) / (sum(res) / 1e3),
                "note": "fh_resample_p_dev: weights + contraction on the resident target fields of "
                        "the timed steps (no fresh target-field step)"}
    phase_ms = leg.phases(max(2, min(args.steps, 3)), flush)
    dominant = max(phase_ms, key=phase_ms.get)
    e2e_times, h2d, d2h = leg.e2e(args.steps, flush)
    e2e_total = max_over_ranks(sum(e2e_times), world, dev)
    contract_tc = (args.precision != "fp64" and bool(leg.tuning["setting"].get("contract_tc"))
                   and 2 * wl.J <= 8192)
    roofs = phase_rooflines(wl, args.precision, phase_ms, leg.stats.get("iters", 0), peaks,
                            contract_tc)
    roof = dict(roofs.get(dominant) or {"bound": "alu", "achieved": None, "peak": None,
                                        "unit": None, "frac": None, "kernel": dominant})
    # (the capture is of the BF16 kernel; the TF32 one updates once per panel)
    roof["traffic"] = MEASURED_TRAFFIC.get(roof.get("kernel")) if args.precision == "bf16" else None
    roof["phase"] = dominant
    roof["phase_ms_per_step"] = phase_ms
    roof["all_phases"] = roofs
    accuracy = {"refine_sweeps_max": leg.stats.get("iters"),
                "refine_residual_max": leg.stats.get("resid")}
    if extra and args.workload == "kite_wide":
        psi_mixed = {j: leg.density(j) for j in WIDE_CHECK_J}
        V_mixed = leg.target_field()[::64]
    tuning = leg.tuning
    leg.close()

    fp64 = other = other_prec = None
    if extra and args.precision != "fp64":
        # ---- the plain FP64 GPU path on the same workload ----
        leg64 = Leg(F, torch, local, stream, wl, "fp64", args)
        per64, _, _ = leg64.timed(args.fp64_steps, 1, flush)
        fp64 = summary(per64, S)
        fp64["phase_ms_per_step"] = leg64.phases(1, flush)
        fp64["tuning"] = leg64.tuning["setting"]
        u64 = leg64.u()
        if args.workload == "kite_wide":
            psi64 = {j: leg64.density(j) for j in WIDE_CHECK_J}
        leg64.close()
        accuracy["u_rel_l2_vs_fp64_gpu"] = rel(u_mixed, u64)
        accuracy["u_max_abs_diff_vs_fp64_gpu"] = float(np.max(np.abs(u_mixed - u64)))
        accuracy["u_compared"] = f"all {n_x} targets x {n_T} times"

        # ---- the other tensor-core precision on the same workload ----
        alt = "tf32" if args.precision == "bf16" else "bf16" if args.precision == "tf32" else None
        if alt:
            la = Leg(F, torch, local, stream, wl, alt, args)
            pa, _, _ = la.timed(max(3, args.steps // 2), 2, flush)
            other_prec = {alt: summary(pa, S)}
            other_prec[alt]["phase_ms_per_step"] = la.phases(1, flush)
            other_prec[alt]["tuning"] = la.tuning["setting"]
            other_prec[alt]["refine_iters"] = la.stats.get("iters")
            other_prec[alt]["u_rel_l2_vs_fp64_gpu"] = rel(la.u(), u64)
            la.close()

        # ---- the other kite workload, both precisions ----
        if args.workload == "kite_wide":
            wl2 = WORKLOADS["kite_pulses"][0]()
            l2 = Leg(F, torch, local, stream, wl2, args.precision, args)
            p2, _, _ = l2.timed(args.steps, args.warmup, flush)
            kp = {"workload": WORKLOADS["kite_pulses"][1], args.precision: summary(p2, wl2.J - 1)}
            kp[args.precision]["tuning"] = l2.tuning["setting"]
            u2 = l2.u()
            l2.close()
            l264 = Leg(F, torch, local, stream, wl2, "fp64", args)
            p264, _, _ = l264.timed(max(args.fp64_steps, 5), 2, flush)
            kp["fp64"] = summary(p264, wl2.J - 1)
            u264 = l264.u()
            l264.close()
            kp["mixed_over_fp64"] = kp[args.precision]["value"] / kp["fp64"]["value"]
            kp["u_rel_l2_vs_fp64_gpu"] = rel(u2, u264)
            other = {"kite_pulses": kp}
        # ---- batching configuration ----
        other = other or {}
        other["star_batch"] = batch_leg(F, torch, local, stream, flush, max(3, args.steps // 4), 2, args.precision)
        # ---- 2D split synthesis (low-frequency quadrature) ----
        other["split_synthesis"] = split_synthesis_leg(F, torch, local, stream, 3, args.precision)
        # ---- serving ----
        other["serving"] = serving_leg([20.0, 100.0], 24, args.precision)

    cpu = None
    if oracle_proc is not None:
        od = finish_oracle(*oracle_proc)
        if od is not None:
            if "kp_u" in od and other and "kite_pulses" in other:
                kp = other["kite_pulses"]
                kp["u_rel_l2_vs_oracle"] = rel(u2, od["kp_u"])
                kp["fp64_u_rel_l2_vs_oracle"] = rel(u264, od["kp_u"])
                kp["u_compared"] = "all 1024 targets x 4096 times"
                kp["oracle_full_step_s"] = float(od["kp_t_step"])
                kp["oracle_solves_per_s"] = (wl2.J - 1) / float(od["kp_t_solve"])
            if "kw_j" in od:
                psi_o = np.split(od["kw_psi"], np.cumsum(od["kw_N"])[:-1])
                errs = {int(j): rel(psi_mixed[int(j)], p) for j, p in zip(od["kw_j"], psi_o)}
                accuracy["psi_rel_l2_vs_oracle"] = errs
                accuracy["psi_rel_l2_vs_oracle_max"] = max(errs.values())
                if fp64:
                    accuracy["fp64_psi_rel_l2_vs_oracle_max"] = max(
                        rel(psi64[int(j)], p) for j, p in zip(od["kw_j"], psi_o))
                Vm = V_mixed[:, od["kw_j"]]
                accuracy["V_rel_l2_vs_oracle"] = rel(Vm, od["kw_V"])
                accuracy["oracle_checked"] = (f"densities at omega_j, j in {list(map(int, od['kw_j']))} "
                                              "(N 64..1920), target fields there at 16 targets")
                # cpu_baseline: the oracle's solves of the sampled frequencies
                c = n3_fit(od["kw_N"], od["kw_t"])
                Nw = wl.N[1:].astype(float)
                est_solves = float(np.sum(c[0] + c[1] * Nw ** 2 + c[2] * Nw ** 3))
                est_step = est_solves + float(od["kw_t_synth16"]) * n_x / 16
                cpu = {"value": len(od["kw_t"]) / float(np.sum(od["kw_t"])), "unit": "solves/s",
                       "cores": int(od["threads"]), "kind": "oracle",
                       "sample": (f"oracle solves at {len(od['kw_t'])} frequencies j in "
                                  f"{list(map(int, od['kw_j']))} (N {int(min(od['kw_N']))}.."
                                  f"{int(max(od['kw_N']))}), {float(np.sum(od['kw_t'])):.1f} s, run "
                                  "in a process beside the GPU legs; solves/s = solves done / time"),
                       "n3_fit_s": {"c0": float(c[0]), "c2": float(c[1]), "c3": float(c[2])},
                       "est_full_step_s": est_step,
                       "est_full_step_note": "N^3 fit over the sampled solves for all 511 solves + "
                                             "spectra and synthesis timed for 16 targets x 4096 "
                                             "times, scaled to 1024 targets (target fields excluded)"}
            if "kp_t_step" in od:
                cpu_full = {"workload": WORKLOADS["kite_pulses"][1], "step_s": float(od["kp_t_step"]),
                            "solves_per_s": 255.0 / float(od["kp_t_step"]),
                            "time_side_s": float(od["kp_t_time_side"]),
                            "note": "the oracle's full step (255 solves, spectra, fields at 1024 "
                                    "targets, synthesis at 4096 times), timed once"}
                if cpu is None:
                    cpu = {"value": cpu_full["solves_per_s"], "unit": "solves/s",
                           "cores": int(od["threads"]), "kind": "oracle", "sample": cpu_full["note"]}
                cpu["full_step_kite_pulses"] = cpu_full

    if rank == 0:
        cfg = {"workload": WORKLOADS[args.workload][1], "precision": args.precision,
               "solves_per_step": S, "time_samples_per_step": n_x * n_T,
               "l2": "flushed between timed steps (256 MiB write)",
               "parallelism": "replicas" if world > 1 else "single GPU"}
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision], "data": "synthetic", "config": cfg,
            "time_samples_per_s": samples_per_s,
            "time_samples_per_s_resident_fields": resident["time_samples_per_s"],
            "resident_fields": resident,
            "p50_ms": float(np.percentile(per_step, 50)),
            "p99_ms": float(np.percentile(per_step, 99)),
            "e2e": {"value": world * S * args.steps / e2e_total, "unit": "solves/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": 1e3 * e2e_total / args.steps},
            "gpu_launches": int(launches),
            "accuracy": accuracy,
            "fp64": fp64,
            "mixed_over_fp64": (value / fp64["value"]) if fp64 else None,
            "other_precisions": other_prec,
            "other_workloads": other,
            "peaks": peaks,
            "tuning": tuning,
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "gb300" and torch.cuda.is_available()) else "gloo"
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        else:
            run_gpu(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
