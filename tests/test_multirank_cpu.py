"""The N > 1 bench path on CPU: two gloo ranks, each an independent replica (no data-path
collective), job time = the maximum over ranks, whole-job throughput = ranks x steps / that time.
Each rank solves its own problem with the oracle; the replicas never exchange data, so every rank's
result equals the single-process result on the same input."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    import datagen
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X, C0 = datagen.small_2d(seed=rank)
    C, rho, info = oracle.solve(X, C0)
    fake_time = 1.0 + rank                  # a slower second replica
    (job,) = bench.max_over_ranks([fake_time], dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, job, info["iters"], C.tobytes()))


def test_two_gloo_replicas_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import datagen
    import oracle
    for rank, job, iters, Cb in out:
        assert job == 2.0                   # the maximum of 1.0 and 2.0
        X, C0 = datagen.small_2d(seed=rank)
        C, _, info = oracle.solve(X, C0)
        assert iters == info["iters"] and Cb == C.tobytes()
    world, steps = 2, 1
    assert world * steps / out[0][1] == 1.0


def test_single_process_max_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.5], None, "cpu") == [3.0, 4.5]
