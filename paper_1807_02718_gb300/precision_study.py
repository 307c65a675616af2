"""Per-result error and solve time of the mixed-precision solvers on the wide-band
kite (512 frequencies on [0, 160], N up to 1920 by 8 points per wavelength, or
forced larger), measured against this library's FP64 path on the same inputs.

    python -m paper_1807_02718_gb300.precision_study [--J 512] [--W 160]
        [--n-force N] [--stride 1] [--precisions tf32,bf16,fp32]

Results (one JSON line per precision): largest relative L2 error over the
frequencies of the densities psi_j and of the target fields V(x, w_j) at 64
targets, relative L2 error of u(x, T) on 64 targets x 4096 times, refinement
sweeps and residual, and the device time of the factorisation and refinement
phases.  --stride s keeps every s-th frequency (smaller device memory for the
FP64 reference at large N); --n-force N makes N grow linearly with the
frequency up to N (rounded to 32) instead of 8 points per wavelength.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import fh_inputs as fi  # noqa: E402

from . import fh as F  # noqa: E402

PREC = {"fp64": F.FH_FP64, "fp32": F.FH_MIXED_FP32, "tf32": F.FH_MIXED_TF32, "bf16": F.FH_MIXED_BF16}


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def run(wl, prec, n_tgt):
    pr = F.Problem(0, PREC[prec])
    pr.discretize(wl.curve, wl.omega, wl.N, wl.c, wl.p)
    pr.solve()                                    # warm-up (allocations)
    F.fh_set_timing(pr.ctx, True)
    F.fh_get_timings(pr.ctx, reset=True)
    st = pr.solve()
    ph = F.fh_get_timings(pr.ctx, reset=True)
    F.fh_set_timing(pr.ctx, False)
    psi = [F.fh_get_density(pr.ctx, j, int(wl.N[j])) for j in range(1, wl.J)]
    pr.window_spectra(wl.a, wl.t0, wl.dt, wl.H)
    xs = wl.x[: 2 * n_tgt]
    u = pr.sample(xs, wl.T)
    V = F.fh_get_target_field(pr.ctx, n_tgt, wl.J)
    out = {"psi": psi, "V": V, "u": u, "iters": st.refine_iters_max, "resid": st.residual_max,
           "factor_ms": ph["factor"]["ms"], "refine_ms": ph["refine"]["ms"]}
    pr.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--J", type=int, default=512)
    ap.add_argument("--W", type=float, default=160.0)
    ap.add_argument("--n-force", type=int, default=None)
    ap.add_argument("--stride", type=int, default=1)
    ap.add_argument("--targets", type=int, default=64)
    ap.add_argument("--precisions", default="tf32,bf16,fp32")
    args = ap.parse_args()
    from . import build
    build.build()
    wl = fi.kite_wide(J=args.J, W=args.W, n_x=args.targets, n_near=3072, n_far=1024,
                      n_force=args.n_force)
    if args.stride > 1:
        # every stride-th frequency as its own (coarser) mesh with the same band
        keep = np.arange(0, wl.J, args.stride)
        wl.omega, wl.N = wl.omega[keep], wl.N[keep]
    ref = run(wl, "fp64", args.targets)
    print(json.dumps({"precision": "fp64", "J": int(wl.J), "max_N": int(wl.N.max()),
                      "factor_ms": ref["factor_ms"]}), flush=True)
    for p in args.precisions.split(","):
        r = run(wl, p, args.targets)
        line = {"precision": p, "J": int(wl.J), "max_N": int(wl.N.max()),
                "psi_rel_l2_max": max(rel(a, b) for a, b in zip(r["psi"], ref["psi"])),
                "V_rel_l2_max": max(rel(r["V"][:, j], ref["V"][:, j]) for j in range(1, wl.J)),
                "u_rel_l2": rel(r["u"], ref["u"]),
                "refine_sweeps_max": r["iters"], "refine_residual_max": r["resid"],
                "factor_ms": r["factor_ms"], "refine_ms": r["refine_ms"],
                "speedup_vs_fp64_solve": ref["factor_ms"] / (r["factor_ms"] + r["refine_ms"])}
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
