"""Seeded synthetic endgame specs and strategy vectors.

This module only draws random numbers and fixes workload parameters; it
holds none of the method's arithmetic (no tree building, no hand ordering,
no payoff computation).  Both the CUDA library's callers and the FP64
oracle's callers take their inputs from here, so the two sides see the same
numbers.

The paper's river endgames (Brains vs AI, Sec. 5) are not available; the
specs below stand in for them with the same shape: a 52-card deck, a public
board, two-card private hands, a strength total order with ties, beliefs per
hand, and a betting skeleton with a handful of pot-fraction bet sizes.

A spec is a plain dict:
    ranks, suits, cards_per_hand, board (card ids, id = rank*suits + suit),
    stack (2), contrib0 (2), bet_frac (list), raise_cap (int, <0 = none),
    allow_allin (bool), strength (int per canonical hand), mu1, mu2
    (float per canonical hand or None for uniform).
Canonical hand order: the deck minus the board in increasing card id; one-card
hands are single cards, two-card hands the pairs (a < b) in lexicographic
order.  Only the number of hands is needed here.
"""
from __future__ import annotations

import math
import numpy as np

HAND_RANKS = 7462  # distinct five-card hand classes; strengths are drawn below it


def num_hands(ranks: int, suits: int, nboard: int, cards_per_hand: int) -> int:
    m = ranks * suits - nboard
    return m if cards_per_hand == 1 else m * (m - 1) // 2


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def tiny_spec(seed: int = 1) -> dict:
    """6-card deck (3 ranks x 2 suits), one card per hand, no board, strength
    = rank, one pot-size bet, at most 2 aggressive actions, contribution 1 and
    100 chips behind each, uniform beliefs."""
    del seed  # fully determined
    ranks, suits = 3, 2
    strength = [c // suits for c in range(ranks * suits)]
    return dict(ranks=ranks, suits=suits, cards_per_hand=1, board=[],
                stack=[100.0, 100.0], contrib0=[1.0, 1.0], bet_frac=[1.0],
                raise_cap=2, allow_allin=False, strength=strength, mu1=None, mu2=None)


def kuhn_spec() -> dict:
    """Kuhn poker: J, Q, K, one card each, ante 1, one bet of 1 chip (half the
    pot of 2), no raise after a bet."""
    return dict(ranks=3, suits=1, cards_per_hand=1, board=[], stack=[1.0, 1.0],
                contrib0=[1.0, 1.0], bet_frac=[0.5], raise_cap=1, allow_allin=False,
                strength=[0, 1, 2], mu1=None, mu2=None)


def fig1_betting() -> dict:
    """Betting parameters of the river skeleton of Fig. 1: $1875 contributed by
    each player, $18125 behind, bets and raises of 3/4 of the pot after
    matching, all-in always available, no raise cap."""
    return dict(stack=[18125.0, 18125.0], contrib0=[1875.0, 1875.0], bet_frac=[0.75],
                raise_cap=-1, allow_allin=True)


def micro_spec(seed: int, ranks: int = 4, suits: int = 2, nboard: int = 2,
               cards_per_hand: int = 2, bet_frac=(0.5, 1.0), raise_cap: int = 2,
               allow_allin: bool = True, stack: float = 6.0, ties: bool = True,
               beliefs: bool = True) -> dict:
    """A small random endgame for brute-force checks."""
    r = _rng(seed)
    board = sorted(r.choice(ranks * suits, size=nboard, replace=False).tolist())
    H = num_hands(ranks, suits, nboard, cards_per_hand)
    top = max(2, H // 2) if ties else 10 * H
    strength = r.integers(0, top, size=H).tolist()
    mu1 = r.uniform(0.5, 1.5, size=H) if beliefs else None
    mu2 = r.uniform(0.5, 1.5, size=H) if beliefs else None
    return dict(ranks=ranks, suits=suits, cards_per_hand=cards_per_hand, board=board,
                stack=[stack, stack], contrib0=[1.0, 1.0], bet_frac=list(bet_frac),
                raise_cap=raise_cap, allow_allin=allow_allin, strength=strength,
                mu1=mu1, mu2=mu2)


def river_spec(seed: int = 2, nboard: int = 5, bet_frac=(0.5, 1.0), raise_cap: int = 3,
               allow_allin: bool = False, stack: float = 200.0, contrib: float = 1.0) -> dict:
    """River-endgame shape: 52-card deck, a seeded board, two-card hands
    (C(47,2) = 1081 for a 5-card board), strengths uniform integers in
    [0, 7462) (ties occur), beliefs uniform in [0.5, 1.5)."""
    r = _rng(seed)
    board = sorted(r.choice(52, size=nboard, replace=False).tolist())
    H = num_hands(13, 4, nboard, 2)
    strength = r.integers(0, HAND_RANKS, size=H).tolist()
    mu1 = r.uniform(0.5, 1.5, size=H)
    mu2 = r.uniform(0.5, 1.5, size=H)
    return dict(ranks=13, suits=4, cards_per_hand=2, board=board,
                stack=[stack, stack], contrib0=[contrib, contrib], bet_frac=list(bet_frac),
                raise_cap=raise_cap, allow_allin=allow_allin, strength=strength,
                mu1=mu1, mu2=mu2)


# The betting abstraction of the paper's experiments (appendix "Libratus'
# betting abstraction"), pot fractions per situation: first action of the
# round, after a check, facing the first bet, facing one raise, facing two
# or more raises.  All-in is always on offer and raises are not capped.  The
# opponent's list has no single-raise entry: its "subsequent raises" list
# serves both raise situations.
LIBRATUS_AI = ([0.25, 0.5, 1.0, 2.0, 4.0, 8.0], [0.25, 0.5, 1.0, 2.0, 4.0, 8.0], [0.4, 0.7, 1.1, 2.0],
               [0.4, 0.7, 2.0], [0.7])
LIBRATUS_OPPONENT = ([0.35, 0.65, 1.0], [0.5, 0.75, 1.0], [0.7, 1.1], [0.7], [0.7])


def libratus_spec(seed: int = 2, ai_player: int = 0, pot: float = 1000.0, total: float = 20000.0,
                  ranks: int = 13, suits: int = 4, nboard: int = 5) -> dict:
    """River endgame with the Libratus betting menus: the AI (`ai_player`)
    and its opponent bet from their own per-situation lists, all-in always
    allowed, no raise cap; each player has put pot/2 in and holds `total`
    chips in all (200 big blinds of 100 at the default).  Deck, board,
    strengths and beliefs as river_spec."""
    r = _rng(seed)
    board = sorted(r.choice(ranks * suits, size=nboard, replace=False).tolist())
    H = num_hands(ranks, suits, nboard, 2)
    strength = r.integers(0, HAND_RANKS, size=H).tolist()
    mu1 = r.uniform(0.5, 1.5, size=H)
    mu2 = r.uniform(0.5, 1.5, size=H)
    menu = [None, None]
    menu[ai_player] = [list(x) for x in LIBRATUS_AI]
    menu[1 - ai_player] = [list(x) for x in LIBRATUS_OPPONENT]
    half = pot / 2.0
    return dict(ranks=ranks, suits=suits, cards_per_hand=2, board=board,
                stack=[total - half, total - half], contrib0=[half, half], bet_frac=[],
                raise_cap=-1, allow_allin=True, menu=menu, strength=strength, mu1=mu1, mu2=mu2)


# Betting menus for the batched workload: (bet fractions, raise cap, all-in,
# stack).  Chosen to cover trees from about ten to about two hundred terminals.
BATCH_MENU = [
    ((1.0,), 2, True, 20.0),
    ((0.5,), 3, False, 200.0),
    ((0.5,), 3, True, 20.0),
    ((0.75,), 4, False, 200.0),
    ((0.5, 1.0), 2, False, 200.0),
    ((0.5, 1.0), 2, True, 30.0),
    ((0.5, 1.0), 3, False, 200.0),
    ((0.33, 0.75), 3, True, 40.0),
    ((0.5, 1.0), 4, False, 200.0),
    ((0.33, 0.66, 1.0), 2, False, 200.0),
    ((0.33, 0.66, 1.0), 2, True, 50.0),
    ((0.33, 0.66, 1.0), 3, False, 200.0),
    ((0.25, 0.5, 1.0), 3, True, 60.0),
    ((0.25, 0.5, 1.0, 2.0), 2, True, 100.0),
]


def batch_specs(seed: int = 4, n: int = 4096, nboard_choices=(3, 4, 5),
                menu_weights=None) -> list:
    """Uneven endgames for one batched launch: board size uniform over
    nboard_choices (1176, 1128, 1081 hands), betting drawn from BATCH_MENU
    with log-spread sizes."""
    r = _rng(seed)
    specs = []
    w = None if menu_weights is None else np.asarray(menu_weights, dtype=np.float64)
    if w is not None:
        w = w / w.sum()
    for _ in range(n):
        nb = int(r.choice(nboard_choices))
        fr, cap, allin, stack = BATCH_MENU[int(r.choice(len(BATCH_MENU), p=w))]
        specs.append(river_spec(seed=int(r.integers(1 << 62)), nboard=nb, bet_frac=fr,
                                raise_cap=cap, allow_allin=allin, stack=stack))
    return specs


def simplex_vectors(nact_per_node, H: int, batch: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Per-infoset uniform-simplex (Dirichlet(1,...,1)) draws in [batch][n][H]
    layout: for every node (in sequence order, its actions consecutive) and
    hand, the node's entries sum to one.  Returned as float64 unless dtype
    is given."""
    r = _rng(seed)
    nact = np.asarray(nact_per_node, dtype=np.int64)
    n = int(nact.sum())
    e = r.exponential(1.0, size=(batch, n, H))
    out = np.empty_like(e)
    s0 = 0
    for na in nact:
        blk = e[:, s0:s0 + na, :]
        out[:, s0:s0 + na, :] = blk / blk.sum(axis=1, keepdims=True)
        s0 += na
    return out.astype(dtype, copy=False)


def integer_vectors(n: int, H: int, batch: int, seed: int, lo: int = -3, hi: int = 4) -> np.ndarray:
    """Small-integer vectors for exact-arithmetic checks."""
    return _rng(seed).integers(lo, hi, size=(batch, n, H)).astype(np.float64)


def turn_spec(seed: int = 2, ranks: int = 13, suits: int = 4, cards_per_hand: int = 2,
              bet_frac_t=(1.0,), raise_cap_t: int = 2, bet_frac_r=(0.5, 1.0), raise_cap_r: int = 2,
              stack: float = 200.0, contrib: float = 1.0, strength_top: int = HAND_RANKS,
              beliefs: bool = True) -> dict:
    """Turn endgame shape: a seeded 4-card board, hands over the remaining
    cards (C(48,2) = 1128 for the full deck), a turn betting round, then a
    river card and a river round.  strength[r][h]: hand h's showdown
    strength with river card r, uniform integers in [0, strength_top) drawn
    independently per card (ties occur); beliefs uniform in [0.5, 1.5)."""
    r = _rng(seed)
    ncard = ranks * suits
    board = sorted(r.choice(ncard, size=4, replace=False).tolist())
    H = num_hands(ranks, suits, 4, cards_per_hand)
    strength = r.integers(0, strength_top, size=(ncard, H))
    mu1 = r.uniform(0.5, 1.5, size=H) if beliefs else None
    mu2 = r.uniform(0.5, 1.5, size=H) if beliefs else None
    return dict(ranks=ranks, suits=suits, cards_per_hand=cards_per_hand, board=board,
                stack=[stack, stack], contrib0=[contrib, contrib],
                bet_frac_t=list(bet_frac_t), raise_cap_t=raise_cap_t, allow_allin_t=False,
                bet_frac_r=list(bet_frac_r), raise_cap_r=raise_cap_r, allow_allin_r=False,
                strength=strength, mu1=mu1, mu2=mu2)

