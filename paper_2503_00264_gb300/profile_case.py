"""Small driver for profiling one kernel of liboci under a profiler.

    python -m paper_2503_00264_gb300.profile_case --case slab3 --sweeps 3
    python -m paper_2503_00264_gb300.profile_case --case multigroup --sweeps 3
    python -m paper_2503_00264_gb300.profile_case --case slab3 --si --sweeps 2
    python -m paper_2503_00264_gb300.profile_case --case batch --slabs 64 --ng 32,4
    python -m paper_2503_00264_gb300.profile_case --case slab3 --precision fp32 --ordering rb --steps 1

Sets up the workload, loads a seeded random iterate and runs exactly --sweeps
sweeps through the C ABI (oci_iterate / si_iterate), then exits.  Prints one
line with the device time of the sweeps (CUDA events).  --case batch runs one
time step of a batch of uneven slabs (J in [1k, 8k]; --ng keeps one (N, G)
class) through oci_batch_step.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2503_00264_gb300 import oci  # noqa: E402
from paper_2503_00264_gb300 import workloads as W  # noqa: E402


def make(case: str, J: int | None):
    if case == "slab3":
        return W.slab_3region(c=0.9, tau=0.1, J=J or 2 ** 18)
    if case == "slab3_ragged":
        return W.slab_3region(c=0.9, tau=0.1, J=J or 2 ** 16, ragged=True)
    if case == "multigroup":
        return W.slab_multigroup(J=J or 2 ** 16)
    raise SystemExit(f"unknown case {case}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="slab3")
    ap.add_argument("--J", type=int, default=None)
    ap.add_argument("--sweeps", type=int, default=3)
    ap.add_argument("--solver", default="structured", choices=["structured", "dense"])
    ap.add_argument("--si", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "tf32", "bf16x3"])
    ap.add_argument("--steps", type=int, default=0, help="run full time steps instead of --sweeps sweeps")
    ap.add_argument("--slabs", type=int, default=64, help="batch: slabs drawn before the --ng filter")
    ap.add_argument("--ng", default=None, help="batch: keep only slabs of this N,G")
    ap.add_argument("--batch-max-iter", type=int, default=200)
    ap.add_argument("--j-hi", type=int, default=8192, help="batch: largest slab (cells)")
    ap.add_argument("--ordering", default="jacobi", choices=["jacobi", "rb"], help="cell ordering of the sweeps")
    a = ap.parse_args()
    import torch
    prec = {"fp64": oci.FP64, "fp32": oci.FP32_IR, "tf32": oci.TF32_IR, "bf16x3": oci.BF16X3_IR}[a.precision]
    if a.case == "batch":
        probs = [b.replace(max_iter=a.batch_max_iter) for b in W.batch_of_slabs(a.slabs, j_lo=1024, j_hi=a.j_hi)]
        if a.ng:
            n_, g_ = (int(x) for x in a.ng.split(","))
            probs = [b for b in probs if (b.N, b.G) == (n_, g_)]
        stream = torch.cuda.Stream()
        with oci.BatchSolver(probs, stream=stream.cuda_stream, precision=prec) as bs:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sts = bs.step(allow_noconv=True)
            e1.record(stream)
            torch.cuda.synchronize()
            its = [st["iters"] for st in sts]
            upd = sum(b.unknowns * k for b, k in zip(probs, its))
            ms = e0.elapsed_time(e1)
            print(f"batch of {len(probs)} slabs ({sum(b.J for b in probs)} cells): sweeps {min(its)}..{max(its)}, "
                  f"{ms:.2f} ms, {upd / ms / 1e6:.1f} G updates/s")
        return
    p = make(a.case, a.J)
    solver = oci.SOLVER_DENSE_LU if a.solver == "dense" else oci.SOLVER_STRUCTURED
    stream = torch.cuda.Stream()
    with oci.Solver(p, solver=solver, precision=prec, stream=stream.cuda_stream) as s:
        if a.ordering == "rb":
            s.set_ordering(oci.ORDER_RED_BLACK)
        print("setup:", s.info())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if a.steps:
            e0.record(stream)
            its = sum((s.si_step() if a.si else s.step())["iters"] for _ in range(a.steps))
            e1.record(stream)
            torch.cuda.synchronize()
            print(f"{p.name}: {a.steps} steps, {its} sweeps, {e0.elapsed_time(e1) / a.steps:.2f} ms/step")
            return
        s.set_psi(W.random_guess(p, 1))
        e0.record(stream)
        (s.si_iterate if a.si else s.iterate)(a.sweeps)
        e1.record(stream)
        torch.cuda.synchronize()
        print(f"{p.name}: {a.sweeps} {'SI' if a.si else 'OCI'} sweeps, {e0.elapsed_time(e1) / a.sweeps * 1e3:.1f} us/sweep")


if __name__ == "__main__":
    main()
