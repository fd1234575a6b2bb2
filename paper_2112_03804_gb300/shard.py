"""Sharding a batch of games over ranks (one GPU each).

Games are independent: a rank builds and solves only its own contiguous
range of the game list (kps_partition balances the ranges by the bytes of
one product, H * (n1 + n2) per game), and the only collective is the final
gather of per-game scalars (exploitabilities, iteration counts) in game
order.  torch.distributed supplies the process group (NCCL on GPUs, gloo on
CPU); nothing on the data path communicates.
"""
from __future__ import annotations

import numpy as np

from . import kps


def game_weights(games) -> np.ndarray:
    """Bytes of one FP32 product per game, H * (n1 + n2) * 4."""
    return np.array([4 * g.info()["H"] * (g.info()["n1"] + g.info()["n2"]) for g in games], dtype=np.int64)


def spec_weights(specs) -> np.ndarray:
    """The same weights, 4 * H * (n1 + n2), from the specs alone (no game is
    built): H from the deck, board and hand size, n1 + n2 from one game on a
    6-card deck per distinct betting configuration (stacks, contributions,
    bet sizes, raise cap, all-in, menu), since the betting tree does not
    depend on the cards."""
    from . import synth
    trees = {}
    out = np.zeros(len(specs), dtype=np.int64)
    for i, s in enumerate(specs):
        menu = s.get("menu")
        key = (tuple(float(v) for v in s["stack"]), tuple(float(v) for v in s["contrib0"]),
               tuple(float(v) for v in s.get("bet_frac", [])), int(s.get("raise_cap", -1)),
               bool(s.get("allow_allin", False)), repr(menu))
        if key not in trees:
            probe = dict(ranks=3, suits=2, cards_per_hand=1, board=[], stack=list(key[0]), contrib0=list(key[1]),
                         bet_frac=list(key[2]), raise_cap=key[3], allow_allin=key[4], menu=menu,
                         strength=[0, 1, 2, 3, 4, 5])
            inf = kps.Game(probe).info()
            trees[key] = inf["n1"] + inf["n2"]
        H = synth.num_hands(int(s["ranks"]), int(s["suits"]), len(s.get("board", [])), int(s["cards_per_hand"]))
        out[i] = 4 * H * trees[key]
    return out


def my_range(weights, rank: int, world: int):
    """[lo, hi) of this rank's games."""
    b = kps.partition(weights, world)
    return int(b[rank]), int(b[rank + 1])


def gather_scalars(local, counts, group=None):
    """All ranks' per-game scalars in game order.  `local` holds this rank's
    values (float64), `counts` the number of games of every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    m = max(int(c) for c in counts) if len(counts) else 0
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    buf = torch.zeros(max(m, 1), dtype=torch.float64, device=dev)
    loc = torch.as_tensor(np.asarray(local, dtype=np.float64))
    buf[:len(loc)] = loc.to(dev)
    out = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(out, buf, group=group)
    return np.concatenate([out[r][:int(counts[r])].cpu().numpy() for r in range(world)])
