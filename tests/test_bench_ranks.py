"""The multi-process path of bench.py on the CPU: two `gloo` ranks, each with
its own replica of the workload (same shape, own seed), reduce their timed
milliseconds by max and their iterations by sum -- the whole-job numbers of a
weak-scaling run.  No data crosses ranks in the solve itself."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

SMALL = dict(n_x=50, L=7, sigma=1.0, support=0.1, noise=0.01, seed=5)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t, it = bench.reduce_over_ranks(10.0 + 5.0 * rank, 400 + rank, dist, torch.device("cpu"))
        prob = bench.replica_problem(SMALL, rank)
        q.put((rank, t, it, float(abs(prob["b"]).sum()), prob["A"]["n"], prob["A"]["m"]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_by_max_and_work_by_sum():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, i0, b0, n0, m0), (r1, t1, i1, b1, n1, m1) = out
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 15.0                 # the slowest rank's time
    assert i0 == i1 == 801.0                # the work of both replicas
    assert (n0, m0) == (n1, m1) and b0 != b1   # same shape, independent data


def test_single_process_keeps_its_own_numbers():
    import bench
    assert bench.reduce_over_ranks(12.5, 400, None, None) == (12.5, 400.0)
