"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank reconstructs its
own replica (no data-path collective); the timing is the maximum over ranks and the reported
value is the whole job's iterations per second.  The oracle arm runs on rank 0 only."""
import io
import os
import socket
import contextlib

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        times = [120.0, 180.0]                    # rank 1 is the slow one
        t = bench.max_over_ranks(times[rank], world, "cpu")
        v = bench.whole_job_value(world, 10, 100, t)
        buf = io.StringIO()
        args = bench.parse_args_list(["--impl", "reference", "--steps", "1", "--warmup", "0"])
        printed = None
        if rank == 1:                             # non-zero ranks of the oracle arm do no work
            with contextlib.redirect_stdout(buf):
                bench.run_reference(args, rank, world)
            printed = buf.getvalue()
        dist.barrier()
        q.put((rank, t, v, printed))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_max_over_ranks_and_whole_job_value_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=100) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, t, v, printed in res:
        assert t == 180.0
        assert abs(v - 2 * 10 * 100 / 0.18) < 1e-9 * v
    assert res[1][3] == ""


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(42.5, 1) == 42.5
    assert bench.whole_job_value(1, 4, 100, 200.0) == 2000.0
