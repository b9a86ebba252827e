"""bench.py's multi-rank host logic with world size 2 on the CPU (gloo,
127.0.0.1): the timed value is the maximum over the ranks, and the
reference arm runs on rank 0 only (the other ranks exit 0 without output)."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench._max_over_ranks(10.0 + 5.0 * rank)
        out.put(("max", rank, got))
        if rank == 1:
            # the reference arm: ranks other than 0 do no work and print nothing
            args = bench.argparse.Namespace(seed=0, ref_sample=1, warmup=0, steps=1, config=2)
            buf = io.StringIO()
            with redirect_stdout(buf):
                rc = bench.run_reference(args)
            out.put(("ref", rank, (rc, buf.getvalue())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rank0_only_reference():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got = [q.get(timeout=10) for _ in range(world + 1)]
    maxes = [v for k, r, v in got if k == "max"]
    assert maxes == [15.0, 15.0]
    ref = [v for k, r, v in got if k == "ref"]
    assert ref == [(0, "")]


def test_unmemoised_oracle_cost_covers_every_size():
    """bench's un-memoised oracle figure: one fresh-memo oracle run per
    distinct subdomain size, projected over the batch by the size counts."""
    sys.path.insert(0, ROOT)
    import bench
    import synth
    prob = synth.elasticity_cubes((3, 1, 1), 2, 3, seed=2)       # sizes 81, 81, 192
    sizes = {}
    for sd in prob.subdomains:
        sizes[sd.K.shape[0]] = sizes.get(sd.K.shape[0], 0) + 1
    out = bench._oracle_unmemoised(prob)
    per = out["s_per_subdomain"]
    assert set(per) == {str(n) for n in sizes} and len(sizes) == 2
    assert abs(out["projected_batch_s"] - sum(per[str(n)] * c for n, c in sizes.items())) <= 1e-12
    assert abs(out["assemblies_per_s"] - len(prob.subdomains) / out["projected_batch_s"]) <= 1e-9
