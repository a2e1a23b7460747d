"""The multi-process (one rank per GPU) bench path on CPU: two gloo ranks,
barrier, max-over-ranks time and the whole-job rate."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    from paper_1808_09571_gb300 import replicas
    dist = replicas.init("gloo")
    ws, r, lr = replicas.env()
    replicas.barrier(dist)
    ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    m = replicas.max_over_ranks(ms, dist)
    out[rank] = (ws, r, lr, m, replicas.job_rate(128, ws, m))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ws, r, lr, m, rate = res[rank]
        assert (ws, r, lr) == (2, rank, rank)
        assert m == 150.0  # both ranks agree on the slowest time
        assert rate == pytest.approx(128 * 2 / 0.150)


def test_single_process_needs_no_group(monkeypatch):
    from paper_1808_09571_gb300 import replicas
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.env() == (1, 0, 0)
    assert replicas.init("gloo") is None
    assert replicas.max_over_ranks(3.5, None) == 3.5
    assert replicas.job_rate(10, 1, 500.0) == 20.0
