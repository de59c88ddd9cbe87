"""Host logic of the N-GPU bench path (replicas: every rank solves its own system),
run as two gloo ranks on the CPU: the job time is the largest per-rank time, the
job's work the sum over ranks, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(dist, 10.0 + rank, "cpu")
    work = bench.sum_over_ranks(dist, 1.5 * (rank + 1), "cpu")
    dist.barrier()
    dist.destroy_process_group()
    # the reference arm: ranks other than 0 leave without work and without output
    rc = None
    if rank != 0:
        class A:
            steps, warmup, gpus = 1, 0, world
        rc = bench.run_reference(A, bench.WORKLOADS["32^3x64-cstar3"], "32^3x64-cstar3")
    out.put((rank, ms, work, rc))


def test_two_rank_aggregation_and_reference_arm():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, work, rc in res:
        assert ms == 11.0 and work == 4.5
    assert res[1][3] == 0


def test_single_process_aggregation():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(None, 3.0, "cpu") == 3.0
    assert bench.sum_over_ranks(None, 2.0, "cpu") == 2.0


def test_all_core_oracle_rate():
    """The all-core CPU baseline: spawned workers, memory-mapped fields, the
    wall time of the parallel region (8^4, a fraction of a second of work)."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_1908_11673_gb300 import workload
    w = bench.WORKLOADS["8^4"]
    U, A = workload.gauge_field(w["L"], w["field_seed"], device="cpu")
    psi = workload.spinor(4096, 1)
    rate, cores, n, wall = bench.oracle_rate_all_cores(w, U, A, psi, 0.05, 0.02)
    assert cores == len(os.sched_getaffinity(0))
    assert 0 < n <= 2048 and wall > 0 and rate > 0
