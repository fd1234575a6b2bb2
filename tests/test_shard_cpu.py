"""Sharding over ranks, on the host: the partitioner and a world-size-2
gloo run of the per-game scalar gather (the only collective)."""
import os

import numpy as np
import pytest

from paper_2112_03804_gb300 import kps, synth


def test_partition_properties():
    r = np.random.default_rng(0)
    for n, parts in ((10, 3), (1, 4), (0, 2), (4096, 8), (7, 7), (5, 1)):
        w = r.integers(1, 1000, size=n)
        b = kps.partition(w, parts)
        assert b[0] == 0 and b[-1] == n and np.all(np.diff(b) >= 0)
        if n:
            sums = np.array([w[b[k]:b[k + 1]].sum() for k in range(parts)])
            assert sums.sum() == w.sum()
            # a prefix split is within one item of the even share
            assert np.max(np.abs(sums - w.sum() / parts)) <= w.max() + 1e-9
    # equal weights split evenly
    assert list(kps.partition(np.ones(8, dtype=np.int64), 4)) == [0, 2, 4, 6, 8]
    with pytest.raises(kps.KpsError):
        kps.partition(np.array([1, -1]), 2)


def test_partition_balances_uneven_games():
    from paper_2112_03804_gb300 import shard
    games = [kps.Game(s) for s in synth.batch_specs(seed=4, n=64)]
    w = shard.game_weights(games)
    b = kps.partition(w, 4)
    sums = np.array([w[b[k]:b[k + 1]].sum() for k in range(4)])
    assert sums.max() <= w.sum() / 4 + w.max()


def _worker(rank, world, port, specs, q):
    import torch.distributed as dist
    from paper_2112_03804_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        games = [kps.Game(s) for s in specs]          # host-only build of every game
        w = shard.game_weights(games)
        lo, hi = shard.my_range(w, rank, world)
        b = kps.partition(w, world)
        counts = np.diff(b)
        # a per-game scalar computed only by the owning rank: nnz of A
        local = [games[i].info()["nnz_A"] for i in range(lo, hi)]
        allv = shard.gather_scalars(local, counts)
        q.put((rank, lo, hi, allv.tolist()))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_gather_in_game_order():
    import socket
    import torch.multiprocessing as mp
    specs = synth.batch_specs(seed=9, n=11)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, specs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (r0, lo0, hi0, v0), (r1, lo1, hi1, v1) = res
    assert lo0 == 0 and hi0 == lo1 and hi1 == 11 and hi0 > 0
    want = [kps.Game(s).info()["nnz_A"] for s in specs]
    assert v0 == want and v1 == want


def _solve_worker(rank, world, port, specs, iters, q):
    import torch.distributed as dist
    from oracle.oracle import OracleGame
    from paper_2112_03804_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = shard.spec_weights(specs)                 # no game built for the split
        b = kps.partition(w, world)
        lo, hi = int(b[rank]), int(b[rank + 1])
        # each rank solves only its own games (RM+, the FP64 oracle) ...
        local = [OracleGame(specs[i]).rmplus(iters)[0] for i in range(lo, hi)]
        # ... and the per-game exploitabilities are the one collective
        allv = shard.gather_scalars(local, np.diff(b))
        q.put((rank, lo, hi, allv.tolist()))
    finally:
        dist.destroy_process_group()


def test_gloo_ranks_solve_their_games_and_gather_exploitabilities():
    import socket
    import torch.multiprocessing as mp
    from oracle.oracle import OracleGame
    specs = [synth.micro_spec(seed=20 + k, ranks=4 + k % 2, nboard=2 + k % 2) for k in range(7)]
    iters = 60
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_solve_worker, args=(r, 2, port, specs, iters, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, lo0, hi0, v0), (_, lo1, hi1, v1) = res
    assert lo0 == 0 and hi0 == lo1 and hi1 == len(specs) and 0 < hi0 < len(specs)
    want = [OracleGame(s).rmplus(iters)[0] for s in specs]
    assert v0 == v1
    assert v0 == want                      # same games, same arithmetic: bit for bit
    assert all(v > 0 for v in want)
