"""The N-rank benchmark path on CPU with the gloo backend (world size 2).

Ranks run independent populations (replicas only: no data-path collective):
the host logic that makes them independent (distinct Philox seeds and
instance ids) and the timing reduction (barrier, max over ranks) run here on
CPU processes; the oracle confirms the ranks' shards are different streams."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle

    ws_, rank_, local = bench.dist_env()
    dist = bench.init_dist(ws_, "gloo")
    t = bench.max_over_ranks(dist, ws_, 1.5 * (rank_ + 1))
    u = bench.sum_over_ranks(dist, ws_, 10.0 * (rank_ + 1))  # site updates of all ranks
    bench.barrier(dist, ws_)
    seed = bench.rank_seed(rank_)
    bases = [bench.rank_instance_base(rank_, i, 4) for i in range(4)]
    r = oracle.pa_run(2, 8, seed, bases[0], 64, oracle.linear_betas(1.0, 3), 2)
    q.put((rank_, t, seed, bases, int(r["sumE"][-1]), r["spins"].tobytes(), u))
    dist.destroy_process_group()


def test_two_ranks_gloo_independent_shards_and_max_timing():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert all(o[1] == 3.0 for o in out)          # max over ranks reached every rank
    assert all(o[6] == 30.0 for o in out)         # whole-job units: the sum over ranks
    assert out[0][2] != out[1][2]                  # distinct seeds
    assert not set(out[0][3]) & set(out[1][3])     # disjoint instance ids
    assert out[0][5] != out[1][5]                  # different populations
