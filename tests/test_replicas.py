"""The multi-rank path of the benchmark on the CPU: independent replicas under
torch.distributed (gloo, world size 2), their seeds, and the whole-job throughput taken
over the slowest rank."""
import socket

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
        out.put((rank, replicas.slowest(secs), replicas.job_throughput(1000.0, secs),
                 replicas.replica_seed(42, rank)))
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
    for rank, slow, thr, seed in res:
        assert slow == 1.5  # the slowest rank's time on every rank
        assert thr == pytest.approx(2 * 1000.0 / 1.5)  # all ranks' units / slowest time
        assert seed == 42 + rank
    assert res[0][3] != res[1][3]  # the replicas draw independent random streams


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
