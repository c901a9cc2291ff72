"""Benchmark of the OCI time step on GB300 (one JSON line on rank 0).

Workload: 2^18-cell slab, S16, one group, 3 repeating regions of 1024 cells with
optical thickness 0.01 / 0.1 / 1, scattering ratio c = 0.9, mean free time
tau = 0.1, unit source, vacuum, tol 1e-10, FP64 (the 2^18-cell config).  A
"step" is one time step: per-step constant, OCI sweeps to convergence on the
device, carry / scalar flux / balance.  Metric: cell-unknown updates per second
= J * 4NG * sweeps / time.

--impl reference times the CPU FP64 oracle on a bounded sample of the same
workload (the host cores of this machine).

Subcommands (measurement tools around the same library; no JSON contract line):
  python bench.py profile --case slab3 --sweeps 3 [--precision fp32] [--ordering rb]
                          [--steps N] [--si] [--solver dense] [--J J]
  python bench.py profile --case batch --slabs 64 --ng 32,4
  python bench.py profile --case table2 --delta2 1.0 --N 16 --dt 10 --steps 1
      one small case for a profiler: set up, run exactly --sweeps sweeps from a
      seeded random iterate (or --steps time steps, or one batched step) and exit
  python bench.py grid [--steps 2] [--json out.json]
      the 2^18-cell slab over c in {0.5, 0.9, 0.99} x tau in {0.01, 0.1, 1, 10}:
      OCI (FP64 Jacobi and red-black, red-black FP32_IR) against SI (scan form)
  python bench.py table2 [--json out.json]
      the paper's GPU experiment (Sec. 3.2, Table 2): OCI and SI seconds per
      converged step over delta_2 x S_N x dt (also in the default run's
      "table2" key)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2503_00264_gb300 import workloads as W  # noqa: E402

METRIC = "OCI cell-unknown updates/s"
UNIT = "updates/s"
SAMPLE_J = 3072
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one FP64 sweep launch on the 2^18-cell S16
# slab (mean of two launches after one warm sweep; the ncu capture of this build summarised in
# profiles/k_oci_sweep_slab3_J262144_S16.md), per (kernel: 0 staged / 1 register form, cells per
# block, angle chunks) the autotuner can pick.  A table of measured constants: it is valid for the
# kernels as built here and is re-taken whenever the sweep kernels change.
SWEEP_DRAM_BYTES_NCU = {
    (0, 64, 2): 272.535552e6 + 99.228544e6,
    (1, 16, 4): 278.423552e6 + 105.256064e6, (1, 16, 8): 278.029312e6 + 106.006912e6,
    (1, 32, 2): 286.496128e6 + 104.577792e6, (1, 32, 4): 278.290304e6 + 104.930688e6,
    (1, 32, 8): 277.979264e6 + 105.660672e6, (1, 64, 2): 285.929216e6 + 105.565184e6,
    (1, 64, 4): 278.013440e6 + 104.868352e6,
}
# FP64 issue rate of one SM: 2 DFMA per clock (GB300: 1.25 TFLOP/s FP64 = 152 SMs x 2 x 2 flops
# x 2.07 GHz); the ALU roofline's peak = SMs x this x 2 flops x the maximum SM clock.
FP64_FMA_PER_SM_CLK = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--c", type=float, default=0.9)
    ap.add_argument("--tau", type=float, default=0.1)
    ap.add_argument("--J", type=int, default=2 ** 18)
    ap.add_argument("--solver", default="structured", choices=["structured", "dense"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-si", action="store_true")
    ap.add_argument("--no-multigroup", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-design-cmp", action="store_true")
    ap.add_argument("--no-fourier", action="store_true")
    ap.add_argument("--no-table2", action="store_true")
    ap.add_argument("--batch-max-iter", type=int, default=600)
    return ap.parse_args()


def workload(args, J=None):
    return W.slab_3region(c=args.c, tau=args.tau, J=J or args.J)


def config(args, p):
    return {"workload": p.name, "J": p.J, "N": p.N, "G": p.G, "c": args.c, "tau": args.tau,
            "regions": "3 x 1024 cells, delta 0.01/0.1/1", "tol": p.tol, "solver": args.solver,
            "l2": "inputs larger than L2: Psi ping-pong + per-step constant = "
                  f"{3 * p.unknowns * 8 / 1e6:.0f} MB per sweep vs 129 MB L2",
            "parallelism": "replicas (independent slabs per rank)"}


def hbm_peak():
    """HBM bandwidth denominator (GB/s) and where it came from: the measured copy
    bandwidth of MEASURED_PEAKS.json when the file is there, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        v = json.load(open(path)).get("hbm_gbs")
        if v:
            return float(v), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampler for the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", str(index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_step_times(p, n, threads):
    """Times (s) and sweeps of n consecutive oracle time steps at `threads` OpenMP threads."""
    import oracle
    oracle.set_threads(threads)
    o = oracle.Oracle(p)
    out = []
    for _ in range(n):
        t0 = time.perf_counter()
        r = o.step()
        out.append((time.perf_counter() - t0, r["iters"]))
    return out


def cpu_baseline(args):
    """The oracle as it stands on the host cores, on the first SAMPLE_J cells of
    the workload (3 regions of 1024 cells): the median of 5 time steps on all
    cores (the reported value) and the median of 3 on one core.  Each step is
    timed from the same state sequence the GPU run starts from (zero initial
    flux); the median step's rate is reported."""
    import oracle
    p = workload(args, SAMPLE_J)
    cores = os.cpu_count() or 1
    allc = _oracle_step_times(p, 5, cores)
    used = oracle.get_threads()
    one = _oracle_step_times(p, 3, 1)
    oracle.set_threads(cores)

    def med(rows):
        rates = sorted(p.unknowns * it / t for t, it in rows)
        return rates[len(rates) // 2]

    return {"value": med(allc), "unit": UNIT, "cores": used, "kind": "oracle",
            "one_thread": {"value": med(one), "unit": UNIT, "cores": 1, "steps": len(one)},
            "sample": f"{SAMPLE_J} cells (3 regions of 1024) of the same slab; median over 5 time steps "
                      f"(all {used} threads; {sum(t for t, _ in allc):.1f} s) and over 3 (one thread; "
                      f"{sum(t for t, _ in one):.1f} s) of the convergence loop"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    p = workload(args, SAMPLE_J)
    o = oracle.Oracle(p)
    for _ in range(args.warmup):
        o.step()
    upd, t_tot = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = o.step()
        t_tot += time.perf_counter() - t0
        upd += p.unknowns * r["iters"]
    v = upd / t_tot
    cores = oracle.get_threads()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config(args, workload(args)), sample_cells=SAMPLE_J,
                           sample=f"each timed step runs the first {SAMPLE_J} cells (3 regions of 1024)"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{SAMPLE_J} cells of the same slab per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2503_00264_gb300 import oci
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    p = workload(args)
    solver = oci.SOLVER_DENSE_LU if args.solver == "dense" else oci.SOLVER_STRUCTURED
    peak_fp64 = oci.fp64_peak()
    s = oci.Solver(p, solver=solver, stream=stream.cuda_stream)
    info64 = s.info()
    smx = None if args.no_mixed else oci.Solver(p, precision=oci.FP32_IR, stream=stream.cuda_stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    for _ in range(args.warmup):
        s.step()
        if smx is not None:
            smx.step()
    # starting state of the timed region, replayed by the end-to-end leg below
    start_pp, start_t = s.state()
    start_psi = s.psi()
    s_start_state, s_start_psi = (start_pp, start_t), start_psi
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = Clocks(local)
    barrier()
    e0.record(stream)
    sweeps, launches = 0, 0
    stats = []
    for _ in range(args.steps):
        st = s.step()
        stats.append(st)
        sweeps += st["iters"]
        launches += 2 + st["iters"] + 2  # step constant + y_c, fused sweeps, carry + balance
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    total_sweeps = sweeps * world  # replicas: every rank does the same work
    value = p.unknowns * total_sweeps / (ms * 1e-3)

    n_sw = 50
    psi_keep = s.psi()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    f0.record(stream)
    s.iterate(n_sw)
    f1.record(stream)
    torch.cuda.synchronize()
    sweep_ms_iter = f0.elapsed_time(f1) / n_sw
    s.set_psi(psi_keep)

    mixed = None
    if smx is not None:
        smx.close()
        mixed = []
        phi64, psi64, b64 = s.phi(), s.psi(), s.balance()
        peaks_hbm, peaks_hbm_src = hbm_peak()
        forms = (("FP32_IR", oci.FP32_IR, "FP32 structured block apply on CUDA cores"),
                 ("TF32_IR", oci.TF32_IR, "TF32 dense block apply on tcgen05 tensor cores"),
                 ("BF16X3_IR", oci.BF16X3_IR, "BF16 hi/lo x3 dense block apply on tcgen05 tensor cores"))
        for name, prec, what in forms:
            sv = oci.Solver(p, precision=prec, stream=stream.cuda_stream)
            for _ in range(args.warmup):
                sv.step()
            m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            clk2 = Clocks(local)
            barrier()
            m0.record(stream)
            mx_sweeps, mx_ref = 0, 0
            for _ in range(args.steps):
                st_mx = sv.step()
                mx_sweeps += st_mx["iters"]
                mx_ref += st_mx["refinements"]
            m1.record(stream)
            barrier()
            clk_mx = clk2.stop()
            mx_ms = max_over_ranks(m0.elapsed_time(m1))
            phimx, psimx, bmx = sv.phi(), sv.psi(), sv.balance()
            info_mx = sv.info()
            sv.close()
            # HBM traffic of the form's step (algorithmic): per inner sweep the FP32
            # operand z, delta_in and delta_out (12 B per unknown; 6 B when two sweeps
            # share one pass over the correction -- the recompute pass at the end of
            # an inner block is not counted); per FP64 refinement (and the initial
            # residual) Psi in/out, c, delta in, z out (32 B per unknown)
            b_sweep = 6 if info_mx["inner_kernel"] in (9, 10, 12) else 12
            step_bytes = (mx_sweeps * b_sweep + (mx_ref + args.steps) * 32) * p.unknowns / args.steps
            step_gbs = step_bytes / (mx_ms / args.steps * 1e-3) / 1e9
            mixed.append({
                "form": name, "block_apply": what,
                "fp64_kept_for": "iterate, residual, norm accumulation, balance tallies, carry",
                "value": p.unknowns * mx_sweeps * world / (mx_ms * 1e-3), "unit": UNIT,
                "ms_per_step": mx_ms / args.steps, "sweeps_per_step": mx_sweeps / args.steps,
                "sweeps_per_step_fp64": sweeps / args.steps,
                "speedup_vs_fp64": (ms / args.steps) / (mx_ms / args.steps),
                "err_vs_fp64": {"phi_rel": float(np.abs(phimx - phi64).max() / np.abs(phi64).max()),
                                "psi_rel": float(np.abs(psimx - psi64).max() / np.abs(psi64).max()),
                                "balance_rel": float(np.abs(bmx - b64).max() / np.abs(b64).max()),
                                "sweeps_diff_total": int(mx_sweeps - sweeps)},
                "refinements_per_step": mx_ref / args.steps,
                "inner_kernel": info_mx["inner_kernel"],
                "inner_shape": {"cells_per_tile": info_mx["cells_per_block"],
                                "angle_chunks": info_mx["angle_chunks"]},
                "hbm": {"bytes_per_step": step_bytes, "achieved_gbs": step_gbs,
                        "peak_gbs": peaks_hbm, "peak_source": peaks_hbm_src, "frac": step_gbs / peaks_hbm,
                        "note": "whole step incl. refinements, FP64 norm/stop rule and carry"}
                if prec == oci.FP32_IR else None,
                "clocks": clk_mx})

    # seconds per converged time step: OCI (FP64 and mixed) against GPU SI
    si_cmp = None
    if not args.no_si:
        si_cmp = []
        for tau in (0.01, 0.1):
            q = W.slab_3region(c=args.c, tau=tau, J=args.J)
            row = {"tau": tau}
            for name, kw, si, mode in (("oci_fp64", {}, False, None), ("oci_fp32ir", {"precision": oci.FP32_IR}, False, None),
                                       ("oci_rb_fp64", {}, False, "rb"),
                                       ("oci_rb_fp32ir", {"precision": oci.FP32_IR}, False, "rb"),
                                       ("si_fp64", {}, True, None), ("si_scan_fp64", {}, True, "scan")):
                with oci.Solver(q, stream=stream.cuda_stream, **kw) as sv:
                    if mode == "rb":
                        sv.set_ordering(oci.ORDER_RED_BLACK)
                    elif mode == "scan":
                        sv.set_si_mode(oci.SI_SCAN)
                    (sv.si_step if si else sv.step)()  # warm step (builds graphs, touches memory)
                    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    nst, its = 2, 0
                    t0e.record(stream)
                    for _ in range(nst):
                        its += (sv.si_step if si else sv.step)()["iters"]
                    t1e.record(stream)
                    torch.cuda.synchronize()
                    row[name] = {"s_per_step": t0e.elapsed_time(t1e) / nst / 1e3, "sweeps_per_step": its / nst}
            row["oci_fp64_speedup_vs_si"] = row["si_fp64"]["s_per_step"] / row["oci_fp64"]["s_per_step"]
            row["oci_fp32ir_speedup_vs_si"] = row["si_fp64"]["s_per_step"] / row["oci_fp32ir"]["s_per_step"]
            row["oci_fp32ir_speedup_vs_si_scan"] = row["si_scan_fp64"]["s_per_step"] / row["oci_fp32ir"]["s_per_step"]
            best_oci = min(row[k]["s_per_step"] for k in ("oci_fp64", "oci_fp32ir", "oci_rb_fp64", "oci_rb_fp32ir"))
            best_si = min(row[k]["s_per_step"] for k in ("si_fp64", "si_scan_fp64"))
            row["best_oci_speedup_vs_best_si"] = best_si / best_oci
            si_cmp.append(row)

    # the paper's cell solve (dense per-cell LU factors applied every sweep, here as
    # our own warp-per-cell kernel) against the structured exact solve, same workload
    design_cmp = None
    if not args.no_design_cmp:
        design_cmp = {}
        for name, solver in (("dense_lu_fp64", oci.SOLVER_DENSE_LU), ("structured_fp64", oci.SOLVER_STRUCTURED)):
            with oci.Solver(p, solver=solver, stream=stream.cuda_stream) as sv:
                sv.set_state(*s_start_state)
                sv.set_psi(s_start_psi)
                t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0e.record(stream)
                st_d = sv.step()
                t1e.record(stream)
                torch.cuda.synchronize()
                ms_d = t0e.elapsed_time(t1e)
                design_cmp[name] = {"ms_per_step": ms_d, "sweeps": st_d["iters"],
                                    "us_per_sweep": 1e3 * ms_d / max(st_d["iters"], 1),
                                    "value": p.unknowns * st_d["iters"] / (ms_d * 1e-3), "unit": UNIT}
        design_cmp["structured_speedup"] = (design_cmp["dense_lu_fp64"]["us_per_sweep"]
                                            / design_cmp["structured_fp64"]["us_per_sweep"])

    # Fourier analysis on the GPU (oci_fourier_rho): rho_OCI and rho_SI of the bench
    # workload's three regions at the mean free times of the SI comparison, and a
    # Table-1-shaped grid (c = 1, S8) with its wall time
    fourier = None
    if not args.no_fourier:
        deltas = np.array([0.01, 0.1, 1.0])
        fourier = {"regions_delta": deltas.tolist(), "c": args.c, "N": p.N, "n_theta": 250, "rho": {}}
        for tau in (0.01, 0.1):
            fourier["rho"][str(tau)] = {
                "oci": oci.fourier_rho(oci.FOURIER_OCI, p.N, deltas, tau, args.c, 250, stream.cuda_stream).tolist(),
                "si": oci.fourier_rho(oci.FOURIER_SI, p.N, deltas, tau, args.c, 250, stream.cuda_stream).tolist()}
        tg, dg = np.meshgrid([0.01, 0.1, 1.0, 10.0, np.inf], [0.01, 0.1, 1.0, 10.0], indexing="ij")
        w0 = time.perf_counter()
        rho_grid = oci.fourier_rho(oci.FOURIER_OCI, 8, dg.ravel(), tg.ravel(), 1.0, 1001, stream.cuda_stream)
        fourier["table1_grid_c1_s8"] = {"tau": [0.01, 0.1, 1.0, 10.0, "inf"], "delta": [0.01, 0.1, 1.0, 10.0],
                                        "rho_oci": rho_grid.reshape(tg.shape).tolist(), "n_theta": 1001,
                                        "seconds": time.perf_counter() - w0}
        # time-march stability map of Sec. 2.2 (Fig. 3's axes: mean free time x cell
        # optical thickness, S16, 75 wave numbers): max |lambda_K| must not exceed 1
        taus_k, dels_k = np.logspace(-3, 3, 25), np.logspace(-3, 2, 21)
        tk, dk = np.meshgrid(taus_k, dels_k, indexing="ij")
        w0 = time.perf_counter()
        lam = oci.fourier_rho(oci.FOURIER_MARCH, 16, dk.ravel(), tk.ravel(), None, 75, stream.cuda_stream)
        fourier["time_march_s16"] = {"tau": taus_k.tolist(), "delta": dels_k.tolist(), "n_theta": 75,
                                     "max_abs_lambda_K": lam.reshape(tk.shape).tolist(),
                                     "sup_abs_lambda_K": float(lam.max()),
                                     "unconditionally_stable": bool(lam.max() <= 1.0 + 1e-12),
                                     "seconds": time.perf_counter() - w0}

    # multigroup slab (G = 8, S16, 2^16 cells): FP64 and the FP32-inner mixed form
    multigroup = None
    if not args.no_multigroup:
        q = W.slab_multigroup()
        multigroup = {"workload": q.name, "J": q.J, "N": q.N, "G": q.G, "unknowns_per_cell": 4 * q.N * q.G}
        for name, kw in (("fp64", {}), ("fp32ir", {"precision": oci.FP32_IR}),
                         ("tf32ir", {"precision": oci.TF32_IR}), ("bf16x3ir", {"precision": oci.BF16X3_IR})):
            with oci.Solver(q, stream=stream.cuda_stream, **kw) as sv:
                sv.step()  # warm step
                t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                nst, its = 2, 0
                t0e.record(stream)
                for _ in range(nst):
                    its += sv.step()["iters"]
                t1e.record(stream)
                torch.cuda.synchronize()
                ms_mg = t0e.elapsed_time(t1e)
                multigroup[name] = {"value": q.unknowns * its / (ms_mg * 1e-3), "unit": UNIT,
                                    "ms_per_step": ms_mg / nst, "sweeps_per_step": its / nst}
                if name == "fp64":
                    phi_mg = sv.phi()
                else:
                    multigroup[name]["phi_rel_vs_fp64"] = float(np.abs(sv.phi() - phi_mg).max() / np.abs(phi_mg).max())

    # batched form: 256 independent slabs (J in [1k, 64k], N in {4..32}, G in {1,4}) in one
    # graph launch per time step; one step, sweeps capped per slab; FP64 and the mixed form
    batched = None
    if not args.no_batched:
        probs = [b.replace(max_iter=args.batch_max_iter) for b in W.batch_of_slabs(256)]
        batched = {"slabs": len(probs), "cells": int(sum(p_.J for p_ in probs)),
                   "unknowns": int(sum(p_.unknowns for p_ in probs)), "max_iter": args.batch_max_iter}
        sample = list(range(0, len(probs), 16))
        phi_b = {}
        for name, prec in (("fp64", oci.FP64), ("fp32_ir", oci.FP32_IR)):
            with oci.BatchSolver(probs, stream=stream.cuda_stream, precision=prec) as bs:
                t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0e.record(stream)
                sts = bs.step(allow_noconv=True)
                t1e.record(stream)
                torch.cuda.synchronize()
                ms_b = t0e.elapsed_time(t1e)
                upd = sum(p_.unknowns * st["iters"] for p_, st in zip(probs, sts))
                ent = {"value": upd / (ms_b * 1e-3), "unit": UNIT, "ms_per_step": ms_b,
                       "converged": int(sum(st["status"] == 0 for st in sts)),
                       "sweeps_min_median_max": [int(np.min([st["iters"] for st in sts])),
                                                 int(np.median([st["iters"] for st in sts])),
                                                 int(np.max([st["iters"] for st in sts]))],
                       "max_balance_rel": float(max(max(st["balance_rel"]) for st in sts if st["status"] == 0))}
                ok = [i for i in sample if sts[i]["status"] == 0]
                if name == "fp64":
                    phi_b = {i: bs.phi(i) for i in ok}
                else:
                    both = [i for i in ok if i in phi_b]
                    ent["phi_rel_vs_fp64_sampled"] = float(max(
                        (np.abs(bs.phi(i) - phi_b[i]).max() / np.abs(phi_b[i]).max() for i in both), default=0.0))
                batched[name] = ent

    # the paper's GPU experiment (Sec. 3.2, Table 2): one converged step of the
    # two-group problem over delta_2 x S_N x dt, OCI (FP64, FP32_IR) against SI
    table2 = None if args.no_table2 else table2_rows(stream)

    # dominant kernel: the fused sweep.  Its average launch duration over the timed
    # region = device time of the K steps / sweeps (an upper bound: includes the
    # per-step constant, carry and balance kernels, < 1 %); cross-checked right
    # after the timed region by n sweeps through oci_iterate (host-launched, so
    # each sweep also waits for the finalize of its predecessor's launch slot)
    sweep_ms = ms / sweeps
    NG = p.N * p.G
    flops_cell = 68 * NG + 32 * p.G * p.G
    bytes_cell = 96 * NG + 4
    flops = flops_cell * p.J
    achieved_tf = flops / (sweep_ms * 1e-3) / 1e12
    # the FP64 sweep kernel and launch shape the autotuner picked for this handle
    sweep_key = (info64["sweep_kernel"], info64["cells_per_block"], info64["angle_chunks"])
    sweep_name = (f"k_oci_sweep_reg<{p.N // info64['angle_chunks']}>" if info64["sweep_kernel"] == 1
                  else "k_oci_sweep_t<0>") + \
        f" (FP64 structured cell solve; {info64['cells_per_block']} cells x {info64['angle_chunks']} angle chunks)"
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    clk_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak_alu = n_sm * FP64_FMA_PER_SM_CLK * 2 * clk_mhz * 1e6
    hbm_pk, hbm_pk_src = hbm_peak()
    hbm_gbs = bytes_cell * p.J / (sweep_ms * 1e-3) / 1e9

    # end to end: the timed region's K steps again from its starting state, with
    # the transport state held on the host: every step uploads psi_prev from
    # pinned memory, solves, and reads psi_prev and phi back (the sweep counts
    # must equal the device-timed ones: same steps, same arithmetic)
    pp_host = torch.from_numpy(start_pp).pin_memory()
    phi_host = torch.zeros((p.J, p.G, 4), dtype=torch.float64).pin_memory()
    s.set_psi(start_psi)
    t_host = start_t
    barrier()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    e2e_sweeps = 0
    for _ in range(args.steps):
        s.set_state(pp_host, t_host)
        st = s.step()
        t_host = s.state_into(pp_host)
        s.phi(phi_host)
        e2e_sweeps += st["iters"]
    g1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(g0.elapsed_time(g1))
    e2e_value = p.unknowns * e2e_sweeps * world / (e2e_ms * 1e-3)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(args, p),
            "sweeps_per_step": sweeps / args.steps,
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peak_alu / 1e12, "unit": "TFLOP/s",
                         "frac": achieved_tf * 1e12 / peak_alu,
                         "traffic": SWEEP_DRAM_BYTES_NCU.get(sweep_key) if (p.J == 2 ** 18 and p.N == 16 and
                                                                             p.G == 1) else None,
                         "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                         "traffic_source": "ncu capture of this kernel and launch shape on the same workload "
                                           "(profiles/k_oci_sweep_slab3_J262144_S16.md); a table of measured "
                                           "constants, not taken in this run",
                         "algorithmic_bytes": bytes_cell * p.J,
                         "kernel": sweep_name,
                         "peak_source": f"derived: {n_sm} SMs x {FP64_FMA_PER_SM_CLK} FP64 FMA/clk x 2 flops x "
                                        f"{clk_mhz:.0f} MHz max SM clock",
                         "peak_measured_dfma_loop": peak_fp64 / 1e12,
                         "frac_of_measured_dfma_loop": achieved_tf * 1e12 / peak_fp64,
                         "sweep_us_oci_iterate": sweep_ms_iter * 1e3,
                         "hbm_achieved_gbs": hbm_gbs, "hbm_peak_gbs": hbm_pk, "hbm_peak_source": hbm_pk_src,
                         "hbm_frac": hbm_gbs / hbm_pk,
                         "sweep_us": sweep_ms * 1e3, "flops_per_cell": flops_cell, "bytes_per_cell": bytes_cell},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": p.J * p.G * p.N * 2 * 8,
                    "sweeps_equal_device_timed": e2e_sweeps == sweeps,
                    "d2h_bytes_per_step": p.J * p.G * p.N * 2 * 8 + p.J * p.G * 4 * 8},
            "gpu_launches": launches,
            "clocks": clocks,
            "precision_forms": mixed,
            "si_comparison": si_cmp,
            "multigroup": multigroup,
            "batched_form": batched,
            "paper_scheme_comparison": design_cmp,
            "fourier": fourier,
            "table2": table2}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- table 2 (Sec. 3.2)
TABLE2_DELTAS = (0.05, 0.1, 0.25, 0.5, 1.0, 2.0, 4.0, 8.0)


def _one_step_ms(p, stream, si=False, precision=None):
    """Device time (CUDA events) of one converged step from the problem's initial
    state, after a warm step from the same state (graphs built, memory touched)."""
    import torch

    from paper_2503_00264_gb300 import oci
    kw = {} if precision is None else {"precision": precision}
    with oci.Solver(p, stream=stream.cuda_stream, **kw) as s:
        pp0, t0 = s.state()
        zero = np.zeros((p.J, p.G, p.N, 4))
        step = s.si_step if si else s.step
        step(allow_noconv=True)
        s.set_state(pp0, t0)
        s.set_psi(zero)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step(allow_noconv=True)
        e1.record(stream)
        torch.cuda.synchronize()
        return {"ms": e0.elapsed_time(e1), "sweeps": st["iters"], "status": st["status"]}


def table2_rows(stream, tol=1e-10, max_iter=200000, verbose=False):
    from paper_2503_00264_gb300 import oci
    rows = []
    for dt in (10.0, 0.1):
        for N in (16, 32):
            if verbose:
                print(f"\n### dt = {dt} (tau_2 = {0.45468 * 0.5 * dt:.4g}), S{N}\n")
                print("| delta_2 | J | OCI sweeps | OCI ms | OCI-FP32IR ms | SI sweeps | SI ms | SI/OCI | SI/OCI-FP32IR |")
                print("|---|---|---|---|---|---|---|---|---|")
            for d in TABLE2_DELTAS:
                p = W.rosa_two_group(d, N, dt).replace(tol=tol, max_iter=max_iter)
                o = _one_step_ms(p, stream)
                m = _one_step_ms(p, stream, precision=oci.FP32_IR)
                si = _one_step_ms(p, stream, si=True)
                row = {"dt": dt, "N": N, "delta2": d, "J": p.J, "oci_fp64": o, "oci_fp32ir": m, "si_fp64": si,
                       "si_over_oci": si["ms"] / o["ms"], "si_over_oci_fp32ir": si["ms"] / m["ms"]}
                rows.append(row)
                if verbose:
                    print(f"| {d} | {p.J} | {o['sweeps']} | {o['ms']:.2f} | {m['ms']:.2f} | {si['sweeps']} | "
                          f"{si['ms']:.2f} | {row['si_over_oci']:.2f} | {row['si_over_oci_fp32ir']:.2f} |", flush=True)
    return rows


def cmd_table2(argv):
    import torch
    ap = argparse.ArgumentParser(prog="bench.py table2")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--max-iter", type=int, default=200000)
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    rows = table2_rows(torch.cuda.Stream(), a.tol, a.max_iter, verbose=True)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(rows, f, indent=1)


# ---------------------------------------------------------------- c x tau grid of the 2^18-cell slab
def cmd_grid(argv):
    import torch

    from paper_2503_00264_gb300 import oci
    ap = argparse.ArgumentParser(prog="bench.py grid")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--J", type=int, default=2 ** 18)
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    stream = torch.cuda.Stream()

    def timed(p, si=False, precision=oci.FP64, red_black=False, scan=False):
        with oci.Solver(p, precision=precision, stream=stream.cuda_stream) as s:
            if red_black:
                s.set_ordering(oci.ORDER_RED_BLACK)
            if scan:
                s.set_si_mode(oci.SI_SCAN)
            step = s.si_step if si else s.step
            step(allow_noconv=True)  # warm step
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sweeps, rho, ok = 0, 0.0, True
            e0.record(stream)
            for _ in range(a.steps):
                st = step(allow_noconv=True)
                sweeps += st["iters"]
                rho = st["rho"]
                ok &= st["status"] == 0
            e1.record(stream)
            torch.cuda.synchronize()
            return {"ms_per_step": e0.elapsed_time(e1) / a.steps, "sweeps_per_step": sweeps / a.steps,
                    "rho_e": rho, "converged": ok}

    rows = []
    print("| c | tau | rho OCI / SI (Fourier, max over regions) | OCI FP64 sweeps / ms | final rho_e | "
          "red-black FP64 sweeps / ms | red-black FP32_IR sweeps / ms | SI sweeps / scan ms | "
          "SI scan / best FP64 OCI | SI scan / best OCI |")
    print("|---|---|---|---|---|---|---|---|---|---|")
    deltas = np.array(W.SLAB3_DELTAS)
    for c in W.SLAB3_C:
        for tau in W.SLAB3_TAU:
            p = W.slab_3region(c=c, tau=tau, J=a.J)
            r_oci = float(oci.fourier_rho(oci.FOURIER_OCI, p.N, deltas, tau, c, 250).max())
            r_si = float(oci.fourier_rho(oci.FOURIER_SI, p.N, deltas, tau, c, 250).max())
            jac = timed(p)
            rb = timed(p, red_black=True)
            rbm = timed(p, precision=oci.FP32_IR, red_black=True)
            si = timed(p, si=True, scan=True)
            best64 = min(jac["ms_per_step"], rb["ms_per_step"])
            best = min(best64, rbm["ms_per_step"])
            row = {"c": c, "tau": tau, "rho_oci": r_oci, "rho_si": r_si, "oci_fp64": jac, "oci_rb_fp64": rb,
                   "oci_rb_fp32ir": rbm, "si_scan": si, "si_over_best_fp64_oci": si["ms_per_step"] / best64,
                   "si_over_best_oci": si["ms_per_step"] / best}
            rows.append(row)
            print(f"| {c} | {tau} | {r_oci:.3f} / {r_si:.3f} | {jac['sweeps_per_step']:.0f} / "
                  f"{jac['ms_per_step']:.1f} | {jac['rho_e']:.3f} | {rb['sweeps_per_step']:.0f} / "
                  f"{rb['ms_per_step']:.1f} | {rbm['sweeps_per_step']:.0f} / {rbm['ms_per_step']:.2f} | "
                  f"{si['sweeps_per_step']:.0f} / {si['ms_per_step']:.2f} | {row['si_over_best_fp64_oci']:.2f} | "
                  f"{row['si_over_best_oci']:.2f} |", flush=True)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(rows, f, indent=1)


# ---------------------------------------------------------------- one small case for a profiler
def cmd_profile(argv):
    import torch

    from paper_2503_00264_gb300 import oci
    ap = argparse.ArgumentParser(prog="bench.py profile")
    ap.add_argument("--case", default="slab3", choices=["slab3", "slab3_ragged", "multigroup", "batch", "table2"])
    ap.add_argument("--delta2", type=float, default=1.0, help="table2: cell width in mean free paths of group 2")
    ap.add_argument("--N", type=int, default=16, help="table2: angles")
    ap.add_argument("--dt", type=float, default=10.0, help="table2: time step")
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
    a = ap.parse_args(argv)
    prec = {"fp64": oci.FP64, "fp32": oci.FP32_IR, "tf32": oci.TF32_IR, "bf16x3": oci.BF16X3_IR}[a.precision]
    stream = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.case == "batch":
        probs = [b.replace(max_iter=a.batch_max_iter) for b in W.batch_of_slabs(a.slabs, j_lo=1024, j_hi=a.j_hi)]
        if a.ng:
            n_, g_ = (int(x) for x in a.ng.split(","))
            probs = [b for b in probs if (b.N, b.G) == (n_, g_)]
        with oci.BatchSolver(probs, stream=stream.cuda_stream, precision=prec) as bs:
            e0.record(stream)
            sts = bs.step(allow_noconv=True)
            e1.record(stream)
            torch.cuda.synchronize()
            its = [st["iters"] for st in sts]
            upd = sum(b.unknowns * k for b, k in zip(probs, its))
            ms_b = e0.elapsed_time(e1)
            print(f"batch of {len(probs)} slabs ({sum(b.J for b in probs)} cells): sweeps {min(its)}..{max(its)}, "
                  f"{ms_b:.2f} ms, {upd / ms_b / 1e6:.1f} G updates/s")
        return
    if a.case == "slab3":
        p = W.slab_3region(c=0.9, tau=0.1, J=a.J or 2 ** 18)
    elif a.case == "slab3_ragged":
        p = W.slab_3region(c=0.9, tau=0.1, J=a.J or 2 ** 16, ragged=True)
    elif a.case == "table2":  # the two-group problem of Sec. 3.2 (J = 100 / delta2 cells)
        p = W.rosa_two_group(a.delta2, a.N, a.dt).replace(tol=1e-10)
    else:
        p = W.slab_multigroup(J=a.J or 2 ** 16)
    solver = oci.SOLVER_DENSE_LU if a.solver == "dense" else oci.SOLVER_STRUCTURED
    with oci.Solver(p, solver=solver, precision=prec, stream=stream.cuda_stream) as s:
        if a.ordering == "rb":
            s.set_ordering(oci.ORDER_RED_BLACK)
        print("setup:", s.info())
        if a.steps:
            e0.record(stream)
            its = sum((s.si_step if a.si else s.step)()["iters"] for _ in range(a.steps))
            e1.record(stream)
            torch.cuda.synchronize()
            print(f"{p.name}: {a.steps} steps, {its} sweeps, {e0.elapsed_time(e1) / a.steps:.2f} ms/step")
            return
        s.set_psi(W.random_guess(p, 1))
        e0.record(stream)
        (s.si_iterate if a.si else s.iterate)(a.sweeps)
        e1.record(stream)
        torch.cuda.synchronize()
        print(f"{p.name}: {a.sweeps} {'SI' if a.si else 'OCI'} sweeps, "
              f"{e0.elapsed_time(e1) / a.sweeps * 1e3:.1f} us/sweep")


def cmd_decompose(argv):
    """The benchmark slab split into contiguous cell ranges over the ranks (the
    spatial decomposition of the paper's Sec. 4 outlook,
    paper_2503_00264_gb300.distributed): every rank sweeps its range with the GPU
    solver -- its interior while the edge values are exchanged, its two end
    blocks after -- and the squared norms are summed every sweep.  Strong
    scaling: the total work is fixed.  Launch one rank per GPU (torchrun, NCCL);
    --backend gloo runs the ranks on one GPU with the exchange through the host.
    Rank 0 prints one JSON line."""
    import torch
    import torch.distributed as dist

    from paper_2503_00264_gb300 import distributed as D
    from paper_2503_00264_gb300 import oci
    ap = argparse.ArgumentParser(prog="bench.py decompose")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--backend", default="nccl", choices=["nccl", "gloo"])
    ap.add_argument("--J", type=int, default=2 ** 18)
    ap.add_argument("--c", type=float, default=0.9)
    ap.add_argument("--tau", type=float, default=0.1)
    ap.add_argument("--no-overlap", action="store_true")
    a = ap.parse_args(argv)
    rank, world, local = dist_env()
    if "MASTER_ADDR" not in os.environ:  # one rank started without a launcher
        import socket
        so = socket.socket()
        so.bind(("127.0.0.1", 0))
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(so.getsockname()[1]), RANK="0", WORLD_SIZE="1")
        so.close()
    torch.cuda.set_device(local if a.backend == "nccl" else 0)
    D.init_process_group(a.backend, timeout_s=600.0)
    p = W.slab_3region(c=a.c, tau=a.tau, J=a.J)
    starts = D.split_cells(p.J, world)
    sub = D.subproblem(p, starts[rank], starts[rank + 1])
    halo = D.HaloExchange(rank, world, p.G, p.N, device="cuda" if a.backend == "nccl" else "cpu")
    stream = torch.cuda.current_stream()
    overlap = not a.no_overlap

    def steps(n):
        its = 0
        for _ in range(n):
            r = D.step(loc, halo, p.inc_left, p.inc_right, p.tol, p.max_iter, overlap=overlap)
            if r["status"] != 0:
                raise RuntimeError(f"rank {rank}: decomposed step ended with status {r['status']}")
            its += r["iters"]
        return its

    with oci.Solver(sub, stream=stream.cuda_stream) as loc:
        steps(a.warmup)
        dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sweeps = steps(a.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        t = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64,
                         device="cuda" if a.backend == "nccl" else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    if rank == 0:
        line = {"metric": METRIC, "value": p.unknowns * sweeps / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
                "scaling": "strong", "dtype": "f64", "data": "synthetic", "mode": "decompose",
                "sweeps_per_step": sweeps / a.steps,
                "config": {"workload": p.name, "J": p.J, "N": p.N, "G": p.G, "c": a.c, "tau": a.tau, "tol": p.tol,
                           "parallelism": f"spatial decomposition over {world} ranks ({a.backend})",
                           "overlap": overlap, "cells_per_rank": [starts[r + 1] - starts[r] for r in range(world)]}}
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


if __name__ == "__main__":
    sub = {"profile": cmd_profile, "grid": cmd_grid, "table2": cmd_table2, "decompose": cmd_decompose}
    if len(sys.argv) > 1 and sys.argv[1] in sub:
        sub[sys.argv[1]](sys.argv[2:])
    else:
        a = parse()
        if a.impl == "reference":
            run_reference(a)
        else:
            run_ours(a)
