"""The N > 1 host logic of bench.py (replicas, one process per GPU) on CPU:
world size 2 over gloo on 127.0.0.1.  Checked: process-group set-up from the
torchrun environment, the barrier, max-over-ranks timing, the whole-job
throughput of weak-scaled replicas, and that the reference arm runs on rank 0
only (other ranks exit 0 without work)."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    try:
        _work(rank, world, port, q)
    except BaseException as e:  # report to the parent instead of hanging it
        import traceback
        q.put((rank, "error", traceback.format_exc()))
        raise


def _work(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    w, r, local = bench._dist_init()
    assert dist.get_backend() == "gloo"
    bench._barrier(w)
    # rank r processed (r + 1) * 1000 units in (r + 1) * 10 ms
    value, ms_max = bench._aggregate(1000.0 * (r + 1), 10.0 * (r + 1), w, "cpu")
    mx = bench._max_over_ranks(float(r), w, "cpu")
    sm = bench._sum_over_ranks(float(r + 1), w, "cpu")

    class A:
        steps, warmup, gpus = 3, 0, world

    ref_rc = bench.run_reference(A) if r == 1 else None  # a non-zero rank returns at once
    bench._barrier(w)
    dist.destroy_process_group()
    q.put((r, w, value, ms_max, mx, sm, ref_rc))


@pytest.mark.timeout(300)
def test_replica_host_logic_world_size_2():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=240) for _ in procs), key=lambda t: t[0])
    errs = [t[2] for t in res if t[1] == "error"]
    assert not errs, errs
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, value, ms_max, mx, sm, ref_rc in res:
        assert w == 2
        assert ms_max == 20.0  # the slowest rank's time
        assert value == pytest.approx(3000.0 / 0.020)  # all units over the slowest time
        assert mx == 1.0 and sm == 3.0
    assert res[1][6] == 0
