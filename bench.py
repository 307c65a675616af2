#!/usr/bin/env python
"""Benchmark of the fast-hybrid 2D scattering path on GB300.

One step = the whole path over one synthetic problem (kite obstacle, 40-pulse
incident train over [0, 400], 256 frequencies on [0, 40], N_j by 8 points per
wavelength (64..480), 1024 targets on r = 3, 4096 times up to T = 1e4):
  a1 nodes/tables -> a2 CFIE assembly -> a3 LU + solve (255 frequency solves)
  -> a4 window spectra (29 windows) -> a5 target fields -> a6 synthesis
  weights -> a7 synthesis contraction.

Headline `value`: frequency solves/s of whole steps with inputs resident in
HBM (device-pointer entry points).  `e2e`: the same through the host-pointer
C-ABI calls, host<->device copies (from and to page-locked host buffers)
included.  Also reported: time samples/s,
per-step p50/p99 latency, the dominant kernel against its roofline, the
oracle timed on the host cores, and SM clocks sampled during the timed
region.  L2 is flushed (256 MiB write) between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--precision fp64|mixed|tf32|bf16]
"""
from __future__ import annotations

import argparse
import json
import math
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
WORKLOAD = "kite_pulses: kite, 40 pulses over [0,400], J=256 on [0,40], N=64..480 (8 ppw), 1024 targets, 4096 times to T=1e4"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="tf32", choices=["fp64", "mixed", "tf32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
    """Complex LU with partial pivoting + one solve: (8/3) N^3 + 8 N^2 real flops."""
    N = np.asarray(N, dtype=np.float64)
    return float(np.sum(8.0 / 3.0 * N ** 3 + 8.0 * N ** 2))


def contract_flops(n_x, n_T, J):
    """u = [Vr|Vi][Gr;Gm]: 2 flops per multiply-add over inner dimension 2J."""
    return 2.0 * n_x * n_T * 2 * J


# Unit-count peaks of one GB300 at its 2070 MHz maximum SM clock: FP64 2 DFMA
# and FP32 128 FFMA per clock per SM (ncu's sustained-peak counters), 152 SMs.
SM_CLOCK_GHZ = 2.07
FP64_PEAK = 2 * 2 * 152 * SM_CLOCK_GHZ * 1e9 / 1e12       # 1.26 TFLOP/s
FP32_PEAK = 128 * 2 * 152 * SM_CLOCK_GHZ * 1e9 / 1e12     # 80.5 TFLOP/s
DF_MAC_INSTR = 11                                          # FP32 instructions per double-float MAC
DF_PEAK = FP32_PEAK / DF_MAC_INSTR                         # FP64-equivalent flop/s of df MACs
TF32_OVER_BF16 = 1.1 / 2.25                                # nominal dense tensor rates

# DRAM bytes (read + write) per step of the kernel as committed, from ncu
# captures of the bench command (--set full, one launch per kernel; both
# launches where the schedule splits a phase into the early and the remaining
# systems).
MEASURED_TRAFFIC = {"field_partial_df_kernel": 2.0e6, "lu_factor_tc_kernel": 384.8e6,
                    "assemble_group_df_kernel": 215.9e6, "contract_df_kernel": 36.6e6}


def window_work(wl):
    """FP64-equivalent flops of the synthesis weights per step: near (t, k):
    4 J x 42 (interpolation from the sampled near sums, J <= 1025) or 4 J h
    (direct paired sinc sums); far (t, k): 4 J R (Horner in the Chebyshev
    ratio); every (t, k): 8 J
    (the B_k accumulation).  R and near/far as in the kernel."""
    J = wl.J
    M = 2 * (J - 1)
    h = M // 2
    W = float(wl.omega[-1])
    span = wl.t0 + wl.dt * (wl.a.size - 1)
    s_k = 15.0 * np.arange(int(np.ceil((span + wl.H) / 15.0)) + 1)
    s_k = s_k[s_k - wl.H < span]
    y = W * (wl.T[:, None] - s_k[None, :]) / np.pi
    near = np.abs(y) < 1.25 * h
    a = np.abs(np.where(near, 2.0 * h, y)) / h
    rho = 1.0 / (a + np.sqrt((a - 1.0) * (a + 1.0)))     # Chebyshev ratio of the far expansion
    R = np.clip(np.ceil(-48 * np.log(2) / np.log(rho)), 1, 64)
    per_near = 4 * J * (SINC_POINTS if J <= SINC_TAB_MAX_J else h)
    return float(np.sum(np.where(near, per_near, 4 * J * R)) + 8 * J * y.size)


SINC_POINTS, SINC_TAB_MAX_J = 42, 1025   # samples per near sum; largest J with the sampled table


OZAKI_PAIRS = 36   # slice pairs (i, j), i + j < 8, of the tensor-core contraction


def phase_rooflines(wl, precision, ms, iters, peaks, contract_tc=False):
    """Achieved against peak per phase: algorithmic work per step (each
    entry's work definition is in its peak_source) over the phase time."""
    N = wl.N[1:].astype(np.float64)
    mixed = precision != "fp64"
    bf16 = peaks.get("bf16_tflops")
    out = {}

    def put(phase, kernel, bound, work, peak, peak_src, unit="TFLOP/s"):
        if ms.get(phase, 0) <= 0 or peak is None:
            return
        ach = work / (ms[phase] * 1e-3) / (1e9 if unit == "GB/s" else 1e12)
        out[phase] = {"kernel": kernel, "bound": bound, "unit": unit, "work_per_step": work,
                      "achieved": ach, "peak": peak, "frac": ach / peak, "peak_source": peak_src}

    fp64_src = "FP64 unit count (2 DFMA/clk/SM x 152 SMs x 2.07 GHz)"
    df_src = "double-float MAC rate: FP32 unit count / 11 instructions per MAC, 2 flop per MAC"
    # the mixed paths run these phases in double-float arithmetic on the FP32
    # pipe: their ceiling is the double-float rate, not the FP64 unit count
    put("assemble", "assemble_group_df_kernel" if mixed else "assemble_group_kernel", "alu",
        100.0 * float(np.sum(N * N)), DF_PEAK if mixed else FP64_PEAK,
        (df_src if mixed else fp64_src) + "; work 1e2 FP64-equivalent flop per entry")
    if precision == "fp64":
        put("factor", "lu_solve_fp64_kernel", "alu", lu_flops(N), FP64_PEAK, fp64_src)
    elif precision == "mixed":
        put("factor", "lu_factor_fp32_kernel", "alu", float(np.sum(8 / 3 * N ** 3)), FP32_PEAK,
            "FP32 unit count (128 FFMA/clk/SM x 152 SMs x 2.07 GHz)")
    else:
        pk = bf16 * (TF32_OVER_BF16 if precision == "tf32" else 1.0) if bf16 else None
        put("factor", "lu_factor_tc_kernel", "tensor", float(np.sum(8 / 3 * N ** 3)), pk,
            "measured bf16 dense GEMM (MEASURED_PEAKS.json)" +
            (" x nominal TF32/BF16 ratio 1.1/2.25" if precision == "tf32" else ""))
    if mixed:
        put("refine", "refine_resid_kernel", "hbm", 24.0 * float(np.sum(N * N)) * max(iters, 1),
            peaks.get("hbm_gbs"), "measured copy bandwidth (MEASURED_PEAKS.json); bytes: the "
            "double-float matrix (16 B/entry, residual) and the FP32 factors (8 B/entry, solves) "
            "per sweep x the largest sweep count", unit="GB/s")
    put("field", "field_partial_df_kernel" if mixed else "field_partial_kernel", "alu",
        50.0 * wl.n_x * float(np.sum(N)), DF_PEAK if mixed else FP64_PEAK,
        (df_src if mixed else fp64_src) + "; work 50 FP64-equivalent flop per (target, node)")
    put("weights", "weights_kernel", "alu", window_work(wl), DF_PEAK, df_src)
    if contract_tc:
        put("contract", "contract_tc_kernel", "tensor", OZAKI_PAIRS * contract_flops(wl.n_x, wl.T.size, wl.J),
            bf16, "measured bf16 dense GEMM (MEASURED_PEAKS.json); work 36 BF16 slice-pair products of "
            "2 n_x n_T (2J) flop (FP64-class result from exact slices)")
    else:
        put("contract", "contract_df_kernel" if mixed else "contract_kernel", "alu",
            contract_flops(wl.n_x, wl.T.size, wl.J), DF_PEAK if mixed else FP64_PEAK,
            "double-float MAC rate: FP32 unit count / 11 instructions per MAC" if mixed else fp64_src)
    return out


# ------------------------------------------------------------ CPU oracle

def oracle_sample_step(wl, n_solve=24, n_tgt=24):
    """The oracle as it stands on a bounded sample of one step, extrapolated to
    the whole step by unit counts.  Returns (est_step_seconds, description)."""
    import oracle as O
    S = wl.J - 1
    js = np.unique(np.linspace(1, wl.J - 1, n_solve).round().astype(int))
    t0 = time.perf_counter()
    psi = {}
    for j in js:
        psi[j] = O.solve_density(wl.curve, int(wl.N[j]) // 2, float(wl.omega[j]), wl.c, wl.p)
    t_solve = time.perf_counter() - t0
    t0 = time.perf_counter()
    s, B = O.window_spectra(wl.a, wl.t0, wl.dt, wl.H, wl.omega)
    t_spec = time.perf_counter() - t0
    xs = wl.x[: 2 * n_tgt]
    t0 = time.perf_counter()
    for j in js:
        O.target_field(wl.curve, int(wl.N[j]) // 2, float(wl.omega[j]), psi[j], xs, wl.c)
    t_field = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    V = rng.standard_normal((n_tgt, wl.J)) + 1j * rng.standard_normal((n_tgt, wl.J))
    t0 = time.perf_counter()
    O.synthesize(B, s, wl.omega, V, wl.T)
    t_syn = time.perf_counter() - t0
    # solves scale with the mix of N^3 actually sampled
    n3 = np.asarray(wl.N[1:], dtype=float) ** 3
    frac = float(np.sum(np.asarray(wl.N[js], dtype=float) ** 3) / np.sum(n3))
    est = (t_solve / frac + t_spec + t_field * (S / len(js)) * (wl.n_x / n_tgt)
           + t_syn * (wl.n_x / n_tgt))
    desc = (f"oracle on {len(js)} of {S} solves (N^3-weighted), window spectra in full, "
            f"target fields for {n_tgt} of {wl.n_x} targets at the sampled frequencies, "
            f"synthesis for {n_tgt} targets x {wl.T.size} times; extrapolated to one step "
            f"(measured {t_solve + t_spec + t_field + t_syn:.1f} s)")
    return est, desc


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """Max of a per-rank scalar over all ranks (identity at world size 1)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


# ----------------------------------------------------------------- arms

def run_reference(args, world, rank):
    if rank != 0:
        return
    wl = fi.kite_pulses()
    S = wl.J - 1
    for _ in range(args.warmup):
        oracle_sample_step(wl, 2, 2)
    ests = []
    desc = ""
    for _ in range(args.steps):
        est, desc = oracle_sample_step(wl)
        ests.append(est)
    total = sum(ests)
    value = S * args.steps / total
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(),
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, world, rank, local):
    import torch
    import torch.distributed as dist
    from paper_1807_02718_gb300 import build
    from paper_1807_02718_gb300 import fh as F

    build.build()
    torch.cuda.set_device(local)
    prec = {"fp64": F.FH_FP64, "mixed": F.FH_MIXED_FP32, "tf32": F.FH_MIXED_TF32,
            "bf16": F.FH_MIXED_BF16}[args.precision]
    wl = fi.kite_pulses()
    S = wl.J - 1
    n_x, n_T = wl.n_x, wl.T.size
    pr = F.Problem(local, prec)
    dev = torch.device("cuda", local)
    # One explicit stream for the library, the L2 flush and the timing events
    # (torch's default stream has the NULL handle, which would leave the
    # library on its own stream, unordered with the events).
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    F.fh_set_stream(pr.ctx, stream.cuda_stream)
    d_a = torch.tensor(wl.a, device=dev, dtype=torch.float64)
    d_x = torch.tensor(wl.x, device=dev, dtype=torch.float64)
    d_T = torch.tensor(wl.T, device=dev, dtype=torch.float64)
    d_u = torch.empty(n_x * n_T, device=dev, dtype=torch.float64)
    flush = torch.empty(256 * 1024 * 1024 // 8, device=dev, dtype=torch.float64)

    # ---- set-up: schedule autotuning on this workload (not timed) ----
    tuning = {"autotuned": False, "setting": F.fh_get_tuning(pr.ctx)}
    if args.tuning:
        F.fh_set_tuning(pr.ctx, **{k: int(v) for k, v in (kv.split("=") for kv in args.tuning.split(","))})
        tuning = {"autotuned": False, "setting": F.fh_get_tuning(pr.ctx)}
    elif not args.no_tune:
        F.fh_discretize(pr.ctx, wl.curve, wl.omega, wl.N, wl.c, wl.p)
        t0 = time.perf_counter()
        chosen, best_ms = F.fh_autotune(pr.ctx, wl.x, reps=3)
        tuning = {"autotuned": True, "setting": chosen, "best_ms": best_ms,
                  "tune_s": time.perf_counter() - t0}

    solve_stats = {}

    def step():
        F.fh_discretize(pr.ctx, wl.curve, wl.omega, wl.N, wl.c, wl.p)
        st = F.fh_solve_frequencies(pr.ctx)
        solve_stats["iters"] = st.refine_iters_max
        solve_stats["resid"] = st.residual_max
        F.fh_window_spectra_dev(pr.ctx, d_a, wl.t0, wl.dt, wl.H)
        F.fh_sample_dev(pr.ctx, d_x, d_T, d_u)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    F.fh_get_timings(pr.ctx, reset=True)

    # ---- device-resident timed region ----
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = []
    for k in range(args.steps):
        flush.fill_(float(k))                      # L2 flush between steps (not timed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    per_step = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(per_step)
    tim = F.fh_get_timings(pr.ctx, reset=True)
    launches = sum(v["launches"] for v in tim.values())
    total_ms = max_over_ranks(total_ms, world, dev)
    value = world * S * args.steps / (total_ms / 1e3)
    samples_per_s = world * n_x * n_T * args.steps / (total_ms / 1e3)

    # ---- per-kernel timing pass (events around each kernel group) ----
    F.fh_set_timing(pr.ctx, True)
    reps = max(2, min(args.steps, 3))
    for k in range(reps):
        flush.fill_(float(k))
        step()
    phases = F.fh_get_timings(pr.ctx, reset=True)
    F.fh_set_timing(pr.ctx, False)
    per_launch = {n: (v["ms"] / v["events"] if v["events"] else 0.0) for n, v in phases.items()}
    step_ms_phases = {n: v["ms"] / reps for n, v in phases.items()}
    dominant = max(step_ms_phases, key=step_ms_phases.get)

    # ---- end to end through the host-pointer API (inputs and u in page-locked host memory) ----
    def pinned(arr):
        return torch.from_numpy(np.ascontiguousarray(arr)).pin_memory().numpy()
    a_p, x_p, T_p, om_p = pinned(wl.a), pinned(wl.x), pinned(wl.T), pinned(wl.omega)
    u_host = torch.empty(n_x * n_T, dtype=torch.float64).pin_memory().numpy()
    e2e_times = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F.fh_discretize(pr.ctx, wl.curve, om_p, wl.N, wl.c, wl.p)
        F.fh_solve_frequencies(pr.ctx)
        F.fh_window_spectra(pr.ctx, a_p, wl.t0, wl.dt, wl.H)
        F.fh_sample(pr.ctx, x_p, T_p, out=u_host)
        e2e_times.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_times)
    e2e_total = max_over_ranks(e2e_total, world, dev)
    assert np.all(np.isfinite(u_host))
    h2d = wl.a.nbytes + wl.x.nbytes + wl.T.nbytes + wl.omega.nbytes + wl.N.nbytes
    d2h = u_host.nbytes

    # ---- rooflines (algorithmic work per step / phase time) ----
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    contract_tc = (args.precision != "fp64" and bool(tuning["setting"].get("contract_tc"))
                   and 2 * wl.J <= 512)
    roofs = phase_rooflines(wl, args.precision, step_ms_phases, solve_stats.get("iters", 0), peaks,
                            contract_tc)
    roof = dict(roofs.get(dominant) or {"bound": "alu", "achieved": None, "peak": None,
                                        "unit": "TFLOP/s", "frac": None, "kernel": dominant})
    roof["traffic"] = MEASURED_TRAFFIC.get(roof.get("kernel"))
    roof["phase"] = dominant
    roof["phase_ms_per_step"] = step_ms_phases
    roof["all_phases"] = roofs
    roof["hbm_peak_gbs"] = peaks.get("hbm_gbs")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        est, desc = oracle_sample_step(wl)
        cpu = {"value": S / est, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": args.precision,
                       "solves_per_step": S, "time_samples_per_step": n_x * n_T,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "time_samples_per_s": samples_per_s,
            "accuracy": {"refine_sweeps_max": solve_stats.get("iters"),
                         "refine_residual_max": solve_stats.get("resid"),
                         "parity": "densities, fields and u within 1e-10 rel L2 of the FP64 oracle "
                                   "(tests/test_parity.py, same precision)"},
            "p50_ms": float(np.percentile(per_step, 50)),
            "p99_ms": float(np.percentile(per_step, 99)),
            "e2e": {"value": world * S * args.steps / e2e_total, "unit": "solves/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "ms_per_step": 1e3 * e2e_total / args.steps},
            "gpu_launches": int(launches),
            "tuning": tuning,
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    pr.close()


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
