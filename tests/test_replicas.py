"""The multi-GPU form of the bench is replicas only: every rank solves its own
independent cluster, no collective touches the data path, and the job's
throughput is all ranks' work over the slowest rank's time (max over ranks).
Checked here with two gloo ranks on the CPU (no GPU involved)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    ws_, r, local, pg = bench.dist_setup(backend="gloo")
    c = bench.replica_cluster("fcc8", r, ws_)
    local_seconds = 1.0 + r  # rank 1 is the slower one
    rate, slowest = bench.job_rate(pg, ws_, 3, local_seconds, "cpu")
    bench.barrier(pg)
    q.put((r, ws_, c.seed, c.M, rate, slowest))
    pg.destroy_process_group()


def test_two_gloo_replicas_take_distinct_clusters_and_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert out[0][2] != out[1][2]  # independent seeded clusters
    assert out[0][3] == out[1][3] == 2457  # the 8x8x8-cell workload of the benchmark
    for o in out:
        assert o[5] == 2.0  # max over ranks
        assert o[4] == pytest.approx(2 * 3 / 2.0)


def test_single_process_needs_no_process_group():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    ws, rank, local, pg = bench.dist_setup()
    assert (ws, rank, pg) == (1, 0, None)
    rate, slowest = bench.job_rate(pg, ws, 4, 2.0, "cpu")
    assert (rate, slowest) == (2.0, 2.0)
