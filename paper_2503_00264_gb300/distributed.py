"""Spatial domain decomposition of one OCI time step across ranks.

Block-Jacobi OCI (Eq. oci) lags all inflow to a cell, so a slab split into
contiguous cell ranges needs, per sweep, only the lagged edge values at each
interface (the paper's Sec. 4 outlook: subdomains exchanging every iteration):
  - rank r receives (Psi_kR, Psi_hR) of the last cell of rank r-1 as its
    incident flux for mu > 0, and (Psi_kL, Psi_hL) of the first cell of rank r+1
    as its incident flux for mu < 0 (2NG values per side per sweep);
  - the squared norms of the ranks' sweeps are summed (one allreduce) and the
    stop rule of Sec. 2.1 is applied to e = sqrt(sum) on every rank.
The iterates are those of single-domain OCI; only the summation order of e
changes.  The local solver is any object with edges(left, right) (fills the
two [G][N][2] buffers), set_boundary(l, r), iterate(1, e_hist) and commit() --
the GPU `oci.Solver`, or a CPU stand-in in tests.  A solver that also has
iterate_part(part, e_out) (the GPU solver: oci_iterate_part) sweeps its
interior cells while the exchange is in flight -- they read no incident flux --
and its two end cells once the halo has arrived.  With a CUDA device (NCCL)
the edge buffers, the received incident fluxes and the norm stay on the GPU:
oci_get_edges writes the send buffers, NCCL moves them, oci_set_boundary reads
the receive buffers, and only the summed e (one scalar per sweep, for the stop
rule) comes to the host.  With gloo they are host tensors.
"""
from __future__ import annotations

import datetime
import math
from typing import Optional

import numpy as np

from . import workloads as W


def split_cells(J: int, world: int):
    """Contiguous cell ranges [starts[r], starts[r+1]) of near-equal size."""
    base, rem = divmod(J, world)
    return [r * base + min(r, rem) for r in range(world + 1)]


def subproblem(prob: W.Problem, a: int, b: int) -> W.Problem:
    """Cells [a, b) of `prob`; the incident fluxes of interior interfaces are set
    each sweep by the exchange."""
    sl = slice(a, b)
    return prob.replace(J=b - a, dx=prob.dx[sl].copy(), mat=prob.mat[sl].copy(),
                        Q=None if prob.Q is None else prob.Q[sl].copy(),
                        psi_init=None if prob.psi_init is None else prob.psi_init[sl].copy(),
                        name=f"{prob.name}[{a}:{b}]")


class RankFailure(RuntimeError):
    """A neighbour did not take part in an exchange within the timeout."""


class HaloExchange:
    """Edge exchange and norm allreduce over torch.distributed (gloo or NCCL),
    with send / receive buffers and the norm kept on `device`."""

    def __init__(self, rank: int, world: int, G: int, N: int, device: str = "cpu"):
        import torch
        self.torch = torch
        self.rank, self.world, self.G, self.N = rank, world, G, N
        self.device = device

        def buf(shape):
            return torch.zeros(shape, dtype=torch.float64, device=device)

        self.send_l, self.send_r = buf((G, N, 2)), buf((G, N, 2))
        self.recv_l, self.recv_r = buf((G, N, 2)), buf((G, N, 2))
        self.e = buf((1,))

    def view(self, t):
        """The buffer as the local solver takes it: the tensor itself on a GPU,
        a numpy view of the same memory on the host."""
        return t.numpy() if t.device.type == "cpu" else t

    def start(self):
        """Post the sends of send_l (to the left neighbour) and send_r (to the
        right one) and the matching receives; return the pending requests."""
        import torch.distributed as dist
        ops = []
        if self.rank > 0:
            ops.append(dist.P2POp(dist.irecv, self.recv_l, self.rank - 1))
            ops.append(dist.P2POp(dist.isend, self.send_l, self.rank - 1))
        if self.rank < self.world - 1:
            ops.append(dist.P2POp(dist.irecv, self.recv_r, self.rank + 1))
            ops.append(dist.P2POp(dist.isend, self.send_r, self.rank + 1))
        try:
            return dist.batch_isend_irecv(ops) if ops else []
        except RuntimeError as e:  # gloo/NCCL timeout or a peer that left
            raise RankFailure(f"rank {self.rank}: edge exchange failed: {e}") from e

    def finish(self, reqs):
        """Wait for the requests of start(); return (inflow from the left
        neighbour, inflow from the right neighbour) as buffers, None at the slab
        ends."""
        try:
            for r in reqs:
                r.wait()
        except RuntimeError as e:
            raise RankFailure(f"rank {self.rank}: edge exchange failed: {e}") from e
        return (self.view(self.recv_l) if self.rank > 0 else None,
                self.view(self.recv_r) if self.rank < self.world - 1 else None)

    def exchange(self):
        """start() and finish() back to back."""
        return self.finish(self.start())

    def allreduce_sum(self, x: float) -> float:
        import torch.distributed as dist
        v = self.torch.tensor([x], dtype=self.torch.float64, device=self.device)
        try:
            dist.all_reduce(v, op=dist.ReduceOp.SUM)
        except RuntimeError as e:
            raise RankFailure(f"rank {self.rank}: norm allreduce failed: {e}") from e
        return float(v.item())

    def norm_of_local(self) -> float:
        """e = sqrt(sum over ranks of e_local^2), e_local in the buffer `e`."""
        import torch.distributed as dist
        v = self.e * self.e
        try:
            dist.all_reduce(v, op=dist.ReduceOp.SUM)
        except RuntimeError as e:
            raise RankFailure(f"rank {self.rank}: norm allreduce failed: {e}") from e
        return math.sqrt(float(v.item()))


def step(local, halo: HaloExchange, inc_left: Optional[np.ndarray], inc_right: Optional[np.ndarray],
         tol: float, max_iter: int, overlap: bool = True) -> dict:
    """One time step of OCI over all ranks; returns dict(status, iters, e, rho).
    overlap: sweep the interior while the edge values are exchanged, where the
    local solver can split a sweep (iterate_part); the iterates are the same."""
    e_prev, rho = 0.0, 0.0
    send_l, send_r, e_buf = halo.view(halo.send_l), halo.view(halo.send_r), halo.view(halo.e)
    split = overlap and hasattr(local, "iterate_part")
    for l in range(max_iter):
        local.edges(send_l, send_r)
        reqs = halo.start()
        if split:
            local.iterate_part(0)  # interior cells: no incident flux read
        from_left, from_right = halo.finish(reqs)
        local.set_boundary(inc_left if from_left is None else from_left,
                           inc_right if from_right is None else from_right)
        if split:
            local.iterate_part(1, e_buf)  # the two end blocks, then e of the whole sweep
        else:
            local.iterate(1, e_buf)
        e = halo.norm_of_local()
        if not math.isfinite(e):
            return dict(status=-6, iters=l + 1, e=e, rho=rho)
        rho = e / e_prev if (l >= 1 and e_prev > 0) else 0.0
        conv = e == 0.0 or (l >= 1 and e < tol * (1.0 - rho))
        e_prev = e
        if conv:
            local.commit()
            return dict(status=0, iters=l + 1, e=e, rho=rho)
    return dict(status=-4, iters=max_iter, e=e_prev, rho=rho)


def init_process_group(backend: str, timeout_s: float = 60.0):
    import torch.distributed as dist
    dist.init_process_group(backend=backend, timeout=datetime.timedelta(seconds=timeout_s))
