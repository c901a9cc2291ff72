"""Full grid of the one-group slab workload: OCI against SI over the scattering
ratio and the mean free time.

The 2^18-cell, 3-region S16 slab (optical thickness per cell 0.01 / 0.1 / 1 in
repeating blocks of 1024 cells) for c in {0.5, 0.9, 0.99} and tau = Sigma_t v dt
in {0.01, 0.1, 1, 10}.  For every point, after one warm step, the mean over the
next time steps of the device time of one converged step (convergence loop,
CUDA events) and of the sweeps per step for:

  - OCI, FP64 structured solve, Jacobi order (the paper's iteration);
  - OCI, FP64 structured solve, red-black order;
  - OCI, FP32 inner sweeps with FP64 refinement, red-black order;
  - SI, FP64, scan form over the cells (the fastest GPU SI here),

with the final rho_e = e_l / e_{l-1} of the OCI FP64 step and the Fourier
spectral radii of OCI and SI (Sec. 2.3; the largest over the three regions),
so that the trend "OCI converges faster as the mean free time shrinks" is read
off measured sweep counts at full size.

    python -m paper_2503_00264_gb300.slab3_sweep [--steps 2] [--json out.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2503_00264_gb300 import oci  # noqa: E402
from paper_2503_00264_gb300 import workloads as W  # noqa: E402

CS = (0.5, 0.9, 0.99)
TAUS = (0.01, 0.1, 1.0, 10.0)


def timed_steps(p, n_steps, si=False, precision=oci.FP64, red_black=False, scan=False):
    import torch
    stream = torch.cuda.Stream()
    with oci.Solver(p, precision=precision, stream=stream.cuda_stream) as s:
        if red_black:
            s.set_ordering(oci.ORDER_RED_BLACK)
        if scan:
            s.set_si_mode(oci.SI_SCAN)
        step = s.si_step if si else s.step
        info = s.info()
        step(allow_noconv=True)  # warm step
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sweeps, rho, ok = 0, 0.0, True
        e0.record(stream)
        for _ in range(n_steps):
            st = step(allow_noconv=True)
            sweeps += st["iters"]
            rho = st["rho"]
            ok &= st["status"] == 0
        e1.record(stream)
        torch.cuda.synchronize()
        return {"ms_per_step": e0.elapsed_time(e1) / n_steps, "sweeps_per_step": sweeps / n_steps,
                "rho_e_last": rho, "converged": bool(ok),
                "kernel": (info["inner_kernel"], info["cells_per_block"], info["angle_chunks"])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--J", type=int, default=2 ** 18)
    ap.add_argument("--max-iter", type=int, default=40000)
    ap.add_argument("--json", default=None)
    a = ap.parse_args()
    deltas = np.array(W.SLAB3_DELTAS)
    rows = []
    for c in CS:
        print(f"\n### c = {c}\n")
        print("| tau | rho OCI / SI (Fourier) | OCI FP64 sweeps | rho_e | OCI FP64 ms | RB FP64 sweeps | RB FP64 ms | "
              "RB FP32_IR sweeps | RB FP32_IR ms | SI sweeps | SI scan ms | SI scan / best FP64 OCI | "
              "SI scan / best OCI |")
        print("|---|---|---|---|---|---|---|---|---|---|---|---|---|")
        for tau in TAUS:
            p = W.slab_3region(c=c, tau=tau, J=a.J).replace(max_iter=a.max_iter)
            r_oci = float(oci.fourier_rho(oci.FOURIER_OCI, p.N, deltas, tau, c).max())
            r_si = float(oci.fourier_rho(oci.FOURIER_SI, p.N, deltas, tau, c).max())
            o = timed_steps(p, a.steps)
            rb64 = timed_steps(p, a.steps, red_black=True)
            rb = timed_steps(p, a.steps, precision=oci.FP32_IR, red_black=True)
            si = timed_steps(p, a.steps, si=True, scan=True)
            best64 = min(o["ms_per_step"], rb64["ms_per_step"])
            best = min(best64, rb["ms_per_step"])
            row = dict(c=c, tau=tau, rho_oci=r_oci, rho_si=r_si, oci_fp64=o, oci_rb_fp64=rb64, oci_rb_fp32ir=rb,
                       si_scan=si, si_over_best_fp64_oci=si["ms_per_step"] / best64,
                       si_over_best_oci=si["ms_per_step"] / best)
            rows.append(row)
            print(f"| {tau} | {r_oci:.3f} / {r_si:.3f} | {o['sweeps_per_step']:.0f} | {o['rho_e_last']:.3f} | "
                  f"{o['ms_per_step']:.1f} | {rb64['sweeps_per_step']:.0f} | {rb64['ms_per_step']:.1f} | "
                  f"{rb['sweeps_per_step']:.0f} | {rb['ms_per_step']:.2f} | "
                  f"{si['sweeps_per_step']:.0f} | {si['ms_per_step']:.2f} | {row['si_over_best_fp64_oci']:.2f} | "
                  f"{row['si_over_best_oci']:.2f} |", flush=True)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
