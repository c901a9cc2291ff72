"""Domain-decomposed OCI over gloo ranks on CPU (world size 2 and 3).

The local solver of every rank is a CPU stand-in built on the oracle, so this
tests the exchange and stop-rule logic of paper_2503_00264_gb300.distributed
without a GPU; the result must equal single-domain OCI."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class OracleLocal:
    """Rank-local solver for tests: the oracle holding one cell range."""

    def __init__(self, prob):
        import oracle
        self.o = oracle.Oracle(prob)

    def edges(self, left, right):
        P = self.o.Psi
        left[...] = P[0][..., [0, 2]]
        right[...] = P[-1][..., [1, 3]]

    def set_boundary(self, il, ir):
        self.o.set_boundary(il, ir)

    def iterate(self, n, e_hist):
        e_hist[:n] = self.o.iterate(n)
        return e_hist

    def commit(self):
        self.o.psi_prev = np.ascontiguousarray(self.o.Psi[..., 2:4])
        self.o.t += self.o.prob.dt


class OracleSplitLocal(OracleLocal):
    """The stand-in with the two-call sweep of the GPU solver (iterate_part):
    the oracle cannot sweep part of a slab, so part 0 only checks the order of
    the calls (it must come between the posting of the exchange and the new
    incident fluxes) and part 1 does the whole sweep."""

    def __init__(self, prob):
        super().__init__(prob)
        self.pending = False
        self.parts = 0

    def set_boundary(self, il, ir):
        assert self.pending, "the incident fluxes must be set between part 0 and part 1"
        super().set_boundary(il, ir)

    def iterate_part(self, part, e_out=None):
        assert self.pending == (part == 1)
        self.pending = part == 0
        self.parts += 1
        if part == 1:
            e = self.o.iterate(1)
            if e_out is not None:
                e_out[:1] = e


def _worker(rank, world, port, seed, steps, fail_rank, q, split=False):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    from paper_2503_00264_gb300 import distributed as D
    from paper_2503_00264_gb300 import workloads as W
    try:
        D.init_process_group("gloo", timeout_s=5.0)
        p = W.random_slab(seed, 37, 8, 2).replace(tol=1e-11)
        starts = D.split_cells(p.J, world)
        sub = D.subproblem(p, starts[rank], starts[rank + 1])
        loc = OracleSplitLocal(sub) if split else OracleLocal(sub)
        halo = D.HaloExchange(rank, world, p.G, p.N)
        res = []
        for k in range(steps):
            if rank == fail_rank and k == 1:
                raise SystemExit(3)  # this rank leaves between steps
            r = D.step(loc, halo, p.inc_left, p.inc_right, p.tol, 5000)
            res.append((r["status"], r["iters"]))
        assert not split or loc.parts == 2 * sum(it for _, it in res)
        q.put((rank, "ok", res, loc.o.Psi.copy()))
    except D.RankFailure as e:
        q.put((rank, "rankfailure", str(e)[:200], None))
    except SystemExit:
        q.put((rank, "left", None, None))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, seed=5, steps=2, fail_rank=-1, split=False):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, seed, steps, fail_rank, q, split))
          for r in range(world)]
    for p in ps:
        p.start()
    out = {}
    for _ in range(world):
        rank, kind, res, psi = q.get(timeout=120)
        out[rank] = (kind, res, psi)
    for p in ps:
        p.join(timeout=30)
    return out


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("world", [2, 3])
def test_domain_decomposed_equals_single_domain(world, split):
    """Single-domain OCI over 2 and 3 ranks, with the plain sweep and with the
    split sweep (interior during the exchange, ends after it)."""
    import oracle
    from paper_2503_00264_gb300 import workloads as W
    p = W.random_slab(5, 37, 8, 2).replace(tol=1e-11)
    o = oracle.Oracle(p)
    ref = [o.step() for _ in range(2)]
    out = _run(world, split=split)
    psi = np.concatenate([out[r][2] for r in range(world)])
    for r in range(world):
        assert out[r][0] == "ok"
        for k in range(2):
            assert out[r][1][k][0] == 0
            assert abs(out[r][1][k][1] - ref[k]["iters"]) <= 1
    assert np.abs(psi - o.Psi).max() <= 1e-11 * np.abs(o.Psi).max()


def test_rank_loss_is_detected_by_timeout():
    """A rank that leaves between steps: its neighbours' next exchange fails
    within the process-group timeout and is reported as RankFailure."""
    out = _run(2, fail_rank=1)
    assert out[1][0] == "left"
    assert out[0][0] == "rankfailure"


def test_split_cells():
    from paper_2503_00264_gb300 import distributed as D
    s = D.split_cells(10, 3)
    assert s == [0, 4, 7, 10]
    assert D.split_cells(5, 5) == [0, 1, 2, 3, 4, 5]
