"""The multi-rank path of bench.py on CPU (gloo, world size 2): the path has
no exchange step (replicas only), so the only cross-rank logic is the job's
time -- the slowest rank's, MAX over ranks -- the whole-job value over all
ranks' frames, and the reference arm running on rank 0 alone."""
import io
import os
import socket
import sys
import types
from contextlib import redirect_stdout

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    local = [100.0, 250.0][rank]
    job = bench.job_time_ms(local, dist)
    value = bench.job_value(8 * 10, ws, job)
    args = types.SimpleNamespace(steps=1, warmup=0, gpus=ws, batch=8)
    out = io.StringIO()
    if rank != 0:   # the reference arm: other ranks return at once, printing nothing
        with redirect_stdout(out):
            bench.reference_arm(args, ws, rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, job, value, out.getvalue()))


def test_max_over_ranks_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, job, value, printed in res:
        assert job == 250.0                           # the slowest rank's time on every rank
        assert abs(value - 2 * 80 / 0.25) < 1e-9      # all ranks' frames over that time
        assert printed == ""
