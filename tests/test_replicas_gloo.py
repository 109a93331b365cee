"""The multi-GPU form (independent replicas, one per rank) on CPU: two gloo ranks time and
combine the way the benchmark does on N GPUs, and seed different instances."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    from paper_2502_14589_gb300 import inputs, replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms, work = replicas.combine(dist, 10.0 + rank, 100.0 * (rank + 1))
        y = inputs.initial_state((8, 8), replicas.instance_seed(rank))
        yb = inputs.initial_state((8, 8), replicas.batch_instance_seed(rank, 3))
        out.put((rank, ms, work, float(y[0]), float(yb[0])))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_benchmark():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_rank_main, args=(world, _free_port(), q), nprocs=world, join=True,
                       start_method="spawn")
    res = sorted(q.get() for _ in range(world))
    for rank, ms, work, _, _ in res:
        assert ms == 11.0                 # the slowest rank's time
        assert work == 300.0              # every rank's work
    assert res[0][3] != res[1][3]         # replicas integrate different instances
    assert res[0][4] != res[1][4]


def test_single_process_combine_is_identity():
    from paper_2502_14589_gb300 import replicas
    assert replicas.combine(None, 3.5, 7.0) == (3.5, 7.0)
    assert replicas.instance_seed(0) == 0


def _failing_rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    from paper_2502_14589_gb300 import replicas
    dist = replicas.init_process_group("gloo", timeout_s=20.0)
    if rank == 1:
        os._exit(3)                       # this rank fails before the timed region ends
    try:
        replicas.combine(dist, 1.0, 1.0)
        q.put((rank, "ok"))
    except Exception as e:                # the survivor learns of it on the host
        q.put((rank, "error: " + type(e).__name__))


def test_a_failed_rank_is_reported_not_waited_for():
    """A rank that dies between barriers turns the other ranks' next collective into an
    error within the process-group timeout (no GPU involved: gloo ranks on the CPU)."""
    import time
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_rank_main, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank was still waiting after 120 s"
    assert procs[1].exitcode == 3
    rank, outcome = q.get()
    assert rank == 0 and outcome.startswith("error"), outcome
    assert time.time() - t0 < 100
