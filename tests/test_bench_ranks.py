"""Multi-rank host logic of bench.py on CPU: two gloo ranks, each with its own step time,
launch count and end-to-end time, must agree on the whole-job figures (max time, summed
launches) and on samples/s = ranks x T / max time (independent chains, weak scaling)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    ms = [10.0, 12.5][rank]
    e2e = [11.0, 10.5][rank]
    launches = [300, 420][rank]
    out = bench.combine_ranks(dist, w, torch.device("cpu"), ms, launches, e2e)
    q.put((r, local, out, bench.job_value(w, 16384, out[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, local, (ms, launches, e2e), value in got:
        assert local == r
        assert ms == 12.5 and e2e == 11.0 and launches == 720
        assert value == pytest.approx(2 * 16384 / 0.0125)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(None, 1, None, 3.5, 7, 4.0) == (3.5, 7, 4.0)
    assert bench.job_value(1, 1000, 2.0) == pytest.approx(500000.0)
