"""The multi-rank path of the benchmark on the CPU: independent replicas under
torch.distributed (gloo, world size 2), their seeds, the whole-job throughput taken over
the slowest rank, and the placement of independent filters on ranks by their HBM need."""
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1605_02406_b300 import replicas


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank)
    try:
        dist.barrier()
        secs = 1.0 + 0.5 * rank  # rank 1 is the slower one
        # independent filters placed by HBM need: the same placement on every rank, each
        # rank counts its own filters' units and the sum reduction gives the whole job
        need = [5.0, 3.0, 3.0, 2.0, 9.0, 1.0]
        where = replicas.place_by_budget(need, world, 10.0)
        mine = sum(n for n, r in zip(need, where) if r == rank)
        out.put((rank, replicas.slowest(secs), replicas.job_throughput(1000.0, secs),
                 replicas.replica_seed(42, rank), tuple(where), replicas.total(mine)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_replicas_combine_over_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get() for _ in range(2))
    for rank, slow, thr, seed, where, tot in res:
        assert slow == 1.5  # the slowest rank's time on every rank
        assert thr == pytest.approx(2 * 1000.0 / 1.5)  # all ranks' units / slowest time
        assert seed == 42 + rank
        assert where == res[0][4]  # one placement, computed alike on both ranks
        # 5 -> 0, 3 -> 1, 3 -> 1 (3 < 5), 2 -> 0 (5 < 6), 9 fits nowhere, 1 -> 1 (6 < 7)
        assert where == (0, 1, 1, 0, -1, 1)
        assert tot == 5.0 + 3.0 + 3.0 + 2.0 + 1.0  # the placed filters' units, summed over ranks
    assert res[0][3] != res[1][3]  # the replicas draw independent random streams


def test_placement_by_budget():
    # one rank: admitted in order while they fit (a later, smaller one may still fit)
    assert replicas.place_by_budget([4, 5, 3, 1], 1, 10) == [0, 0, -1, 0]
    # least-loaded rank that fits; ties go to the lowest rank
    assert replicas.place_by_budget([4, 4, 1, 1, 6], 3, 6) == [0, 1, 2, 2, -1]
    rng = np.random.default_rng(3)
    need = rng.uniform(0.5, 4.0, 200).tolist()
    for world in (1, 2, 5, 8):
        where = replicas.place_by_budget(need, world, 30.0)
        load = np.zeros(world)
        for n, r in zip(need, where):
            if r >= 0:
                load[r] += n
        assert (load <= 30.0 + 1e-12).all()
        # a rejected filter fits on no rank at the moment it is considered
        used = np.zeros(world)
        for n, r in zip(need, where):
            if r < 0:
                assert (used + n > 30.0).all()
            else:
                assert used[r] == used[[k for k in range(world) if used[k] + n <= 30.0]].min()
                used[r] += n


def test_single_process_is_its_own_job(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.rank_env() == (1, 0, 0)
    assert replicas.slowest(2.5) == 2.5
    assert replicas.job_throughput(10.0, 2.0) == 5.0
    monkeypatch.setenv("WORLD_SIZE", "4")
    monkeypatch.setenv("RANK", "3")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert replicas.rank_env() == (4, 3, 1)
