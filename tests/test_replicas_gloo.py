"""Host-side multi-rank logic (replicas only) with two gloo ranks on CPU:
max/sum reductions over ranks, round-robin sharding of ensembles and
request streams (every item exactly once), distinct per-rank seeds."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

from paper_2508_16639_gb300 import replicas as R  # noqa: E402
from paper_2508_16639_gb300 import workloads as W  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = R.rank_info()
        dist.barrier()
        mx = R.max_over_ranks(1.5 + r, dist)
        sm = R.sum_over_ranks(10.0 * (r + 1), dist)
        reps = W.ensemble(37, seed=4)
        mine = [x["index"] for x in R.shard(reps, r, w)]
        seed = R.replica_seed(W.SEED0, r)
        q.put((r, w, lr, mx, sm, mine, seed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    assert all(o[3] == 2.5 for o in out)            # max over ranks
    assert all(o[4] == 30.0 for o in out)           # sum over ranks
    allidx = sorted(out[0][5] + out[1][5])
    assert allidx == list(range(37))                # every replica exactly once
    assert abs(len(out[0][5]) - len(out[1][5])) <= 1
    assert out[0][6] != out[1][6]                   # independent lattices


def test_single_process_fallbacks():
    assert R.max_over_ranks(3.0) == 3.0 and R.sum_over_ranks(2.0) == 2.0
    assert R.shard(range(5), 0, 1) == [0, 1, 2, 3, 4]
    with pytest.raises(ValueError):
        R.shard(range(5), 2, 2)
