"""Host logic of the batched solve (no GPU): the LPT plan of sl_batch_plan and the sharding of
instances over ranks, including a two-rank gloo run."""
import os

import numpy as np
import pytest

import workloads as W


def _lib():
    import paper_1605_04821_gb300 as S
    S.load()
    return S


def _lpt_reference(cost, bins):
    """Longest processing time first: decreasing cost (ties by index), least-loaded bin
    (ties by the lowest bin)."""
    order = sorted(range(len(cost)), key=lambda i: (-cost[i], i))
    load = [0.0] * bins
    out = [0] * len(cost)
    for i in order:
        b = min(range(bins), key=lambda w: (load[w], w))
        out[i] = b
        load[b] += cost[i]
    return out


@pytest.mark.parametrize("n,bins,seed", [(1, 1, 0), (7, 3, 1), (256, 16, 2), (40, 64, 3), (100, 4, 4)])
def test_plan_is_lpt(n, bins, seed):
    S = _lib()
    rng = np.random.default_rng(seed)
    cost = rng.integers(1, 20, n).astype(float)  # integer costs: many ties
    plan = S.lpt_plan(cost, bins)
    assert list(plan) == _lpt_reference(list(cost), bins)
    load = np.bincount(plan, weights=cost, minlength=bins)
    # list-scheduling guarantee: makespan <= average load + largest item
    assert load.max() <= cost.sum() / bins + cost.max() + 1e-9


def test_plan_rejects_bad_arguments():
    S = _lib()
    with pytest.raises(S.SLError):
        S.lpt_plan([1.0, 2.0], 0)


def test_shards_cover_every_instance_once():
    S = _lib()
    probs = W.batched(n_inst=64, seed=1, sizes=(9, 17), k_range=(3, 9), n_steps=2)
    parts = [S.shard(probs, 3, r) for r in range(3)]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(64))
    costs = [sum(S.instance_cost(probs[i]) for i in p) for p in parts]
    assert max(costs) - min(costs) <= max(S.instance_cost(p) for p in probs)


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import paper_1605_04821_gb300 as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    S.load()
    probs = W.batched(n_inst=32, seed=2, sizes=(9, 17), k_range=(3, 9), n_steps=2)
    mine = S.shard(probs, world, rank)
    got = [None] * world
    dist.all_gather_object(got, mine)   # host-side gather of the results' indices
    dist.destroy_process_group()
    q.put((rank, got))


def test_two_rank_gloo_sharding():
    import multiprocessing as mp
    import socket
    ctx = mp.get_context("spawn")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, got in res:
        flat = sorted(i for part in got for i in part)
        assert flat == list(range(32))
        assert set(got[0]).isdisjoint(got[1])
    assert res[0][1] == res[1][1]
