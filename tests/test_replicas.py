"""The replica path of the benchmark on the host: two gloo ranks on CPU find
their rank from the torchrun environment, agree on the slowest rank's time,
and report the whole-job rate (units of all ranks over that time)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    from paper_1208_3210_gb300 import replicas
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    r, lr, w = replicas.rank_info()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        # rank r "took" 1 + r seconds; every rank must see the largest
        t = replicas.max_over_ranks(1.0 + r, w, "cpu")
        rate = replicas.whole_job_rate(1000, w, 10, t)
        q.put((r, lr, w, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    out = sorted(q.get(timeout=10) for _ in range(world))
    for r, (rank, local_rank, w, t, rate) in enumerate(out):
        assert (rank, local_rank, w) == (r, r, world)
        assert t == pytest.approx(2.0)                       # the slower rank
        assert rate == pytest.approx(1000 * 2 * 10 / 2.0)    # both ranks' units


def test_single_rank_defaults(monkeypatch):
    from paper_1208_3210_gb300 import replicas
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.rank_info() == (0, 0, 1)
    assert replicas.max_over_ranks(3.5, 1) == 3.5
    assert replicas.whole_job_rate(8, 1, 4, 2.0) == pytest.approx(16.0)
