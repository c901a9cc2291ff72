"""Domain-decomposed OCI (the paper's Sec. 4 outlook) with the GPU solver as
every rank's local solver: two gloo ranks, each a process holding an
oci.Solver for its cell range on the one GPU of this machine.  The ranks'
kernels never wait on one another -- the edge values and the norm go through
the host between launches -- so sharing one GPU is safe.  The result must be
single-domain OCI: the oracle's sweep counts within one (the norm is summed in
another order) and the same flux within 1e-12."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, seed, J, N, G, steps, q, overlap=True):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    from paper_2503_00264_gb300 import distributed as D
    from paper_2503_00264_gb300 import oci
    from paper_2503_00264_gb300 import workloads as W
    try:
        torch.cuda.set_device(0)
        D.init_process_group("gloo", timeout_s=60.0)
        p = W.random_slab(seed, J, N, G).replace(tol=1e-11)
        starts = D.split_cells(p.J, world)
        sub = D.subproblem(p, starts[rank], starts[rank + 1])
        halo = D.HaloExchange(rank, world, p.G, p.N)
        res = []
        with oci.Solver(sub, stream=torch.cuda.current_stream().cuda_stream) as loc:
            for _ in range(steps):
                r = D.step(loc, halo, p.inc_left, p.inc_right, p.tol, 5000, overlap=overlap)
                res.append((r["status"], r["iters"]))
            q.put((rank, "ok", res, loc.psi(), loc.phi()))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, f"error: {e!r}"[:300], None, None, None))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


@pytest.mark.parametrize("overlap", [True, False])
@pytest.mark.parametrize("seed,J,N,G", [(7, 301, 8, 2), (8, 1000, 16, 1)])
def test_decomposed_gpu_solver_equals_single_domain_oracle(seed, J, N, G, overlap):
    """With overlap every rank sweeps its interior (oci_iterate_part 0) while
    the edge values are in flight and its two end blocks after they arrive."""
    import multiprocessing as mp

    import oracle
    from paper_2503_00264_gb300 import workloads as W
    world, steps = 2, 2
    p = W.random_slab(seed, J, N, G).replace(tol=1e-11)
    o = oracle.Oracle(p)
    ref = [o.step() for _ in range(steps)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, seed, J, N, G, steps, q, overlap))
          for r in range(world)]
    for pr in ps:
        pr.start()
    out = {}
    for _ in range(world):
        rank, kind, res, psi, phi = q.get(timeout=300)
        out[rank] = (kind, res, psi, phi)
    for pr in ps:
        pr.join(timeout=60)
    for r in range(world):
        assert out[r][0] == "ok", out[r][0]
        for k in range(steps):
            assert out[r][1][k][0] == 0
            assert abs(out[r][1][k][1] - ref[k]["iters"]) <= 1, (r, k, out[r][1][k], ref[k]["iters"])
    psi = np.concatenate([out[r][2] for r in range(world)])
    phi = np.concatenate([out[r][3] for r in range(world)])
    assert np.abs(psi - o.Psi).max() <= 1e-11 * np.abs(o.Psi).max()
    assert np.abs(phi - ref[-1]["phi"]).max() <= 1e-12 * np.abs(ref[-1]["phi"]).max()


def test_bench_decompose_mode_two_ranks_on_one_gpu():
    """bench.py decompose launched by torchrun as two gloo ranks on the one GPU:
    one JSON line from rank 0 whose sweeps per step are those of the
    single-domain solver within one (only the norm's summation order differs)."""
    import json
    import subprocess
    import sys

    from paper_2503_00264_gb300 import oci
    from paper_2503_00264_gb300 import workloads as W
    J, steps = 4096, 2
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "decompose", "--backend", "gloo", "--J", str(J), "--steps", str(steps), "--warmup", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["scaling"] == "strong" and d["mode"] == "decompose" and d["value"] > 0
    assert d["config"]["overlap"] is True and d["config"]["cells_per_rank"] == [J // 2, J // 2]
    p = W.slab_3region(c=0.9, tau=0.1, J=J)
    with oci.Solver(p) as s:
        its = [s.step()["iters"] for _ in range(1 + steps)][1:]
    assert abs(d["sweeps_per_step"] - sum(its) / steps) <= 1.0, (d["sweeps_per_step"], its)
