"""Runtime sweep of the paper's GPU experiment (Sec. 3.2, Table 2, Figs. 6-7).

Two-group problem of Table 2: L = 100 cm, vacuum on both sides, psi0 = 0,
Q = 1, group 2 optical thickness delta_2 = Sigma_2 dx swept, S_N in {16, 32},
dt in {0.1, 10} (group-2 mean free time 0.0227 and 2.2734).  For every point
the wall time of one converged time step (convergence loop only, CUDA events,
as the paper times it) is measured for OCI (FP64 structured solve, and the
mixed FP32-inner form) and for SI (FP64), with the sweep counts.

    python -m paper_2503_00264_gb300.table2_sweep [--tol 1e-10] [--json out.json]

Prints one markdown table per (dt, N).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2503_00264_gb300 import oci  # noqa: E402
from paper_2503_00264_gb300 import workloads as W  # noqa: E402

DELTAS = (0.05, 0.1, 0.25, 0.5, 1.0, 2.0, 4.0, 8.0)


def one_step(p, si=False, precision=oci.FP64):
    import torch
    stream = torch.cuda.Stream()
    with oci.Solver(p, precision=precision, stream=stream.cuda_stream) as s:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = (s.si_step if si else s.step)(allow_noconv=True)
        e1.record(stream)
        torch.cuda.synchronize()
        return {"ms": e0.elapsed_time(e1), "sweeps": st["iters"], "status": st["status"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--max-iter", type=int, default=200000)
    ap.add_argument("--json", default=None)
    a = ap.parse_args()
    # warm the context and the kernels once
    one_step(W.rosa_two_group(1.0, 16, 0.1).replace(tol=a.tol))
    rows = []
    for dt in (10.0, 0.1):
        for N in (16, 32):
            print(f"\n### dt = {dt} (tau_2 = {0.45468 * 0.5 * dt:.4g}), S{N}\n")
            print("| delta_2 | J | OCI sweeps | OCI ms | OCI-FP32IR ms | SI sweeps | SI ms | SI/OCI | SI/OCI-FP32IR |")
            print("|---|---|---|---|---|---|---|---|---|")
            for d in DELTAS:
                p = W.rosa_two_group(d, N, dt).replace(tol=a.tol, max_iter=a.max_iter)
                o = one_step(p)
                m = one_step(p, precision=oci.FP32_IR)
                s = one_step(p, si=True)
                row = dict(dt=dt, N=N, delta2=d, J=p.J, oci=o, oci_fp32ir=m, si=s,
                           si_over_oci=s["ms"] / o["ms"], si_over_oci_fp32ir=s["ms"] / m["ms"])
                rows.append(row)
                print(f"| {d} | {p.J} | {o['sweeps']} | {o['ms']:.2f} | {m['ms']:.2f} | {s['sweeps']} | "
                      f"{s['ms']:.2f} | {row['si_over_oci']:.2f} | {row['si_over_oci_fp32ir']:.2f} |", flush=True)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
