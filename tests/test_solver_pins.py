"""Pins for the oracle's solver schedules (RM+ and Discounted CFR).

Every GPU solver test is judged against oracle/kps_oracle.c's RM+ and DCFR
loops iterate by iterate, so those loops are pinned here, independently of
their sequence-form code, by a textbook counterfactual-regret walk of Kuhn
poker's game tree written in this file (chance deals the cards, histories
are action strings, no matrices), run with the schedule the solver reading
states (Sec. 2 first-order methods; Sec. 5 runs DCFR):

  RM+   iteration t: add t * x_t to player 1's average, update player 1's
        regrets R <- max(0, R + q - v) against y_t, regret-match; add t * y_t
        to player 2's average, update player 2 against the NEW x_{t+1}.
  DCFR  the same order; R <- (R + q - v) * t^a / (t^a + 1) if that sum is
        positive, else * t^b / (t^b + 1); regret matching on positive parts;
        weight t^g in the averages; (a, b, g) = (1.5, 0, 2).

A plausible slip anywhere (uniform instead of linear averaging, averaging
the strategy after the update, simultaneous instead of alternating updates,
a weight t + 1, swapped discount exponents, a discount from t - 1) changes
the averages after two to six iterations, so the walk is compared with the
oracle's averages after every one of t = 1..6 iterations.

The walk itself is pinned by values worked out by hand for Kuhn poker
(ante 1, bet 1, J < Q < K, each ordered deal with probability 1/6), starting
from uniform play.  Player 1, iteration 1, counterfactual values
(chance x opponent reach x payoff, summed over the two deals):
  J at the root: check 2/6 (1/2 (-1) + 1/2 (1/2 (-1) + 1/2 (-2))) = -5/12,
                 bet   2/6 (1/2 (+1) + 1/2 (-2)) = -1/6, value -7/24,
                 regrets (0, 1/8);
  J facing check-bet: fold 2/6 1/2 (-1) = -1/6, call 2/6 1/2 (-2) = -1/3,
                 value -1/4, regrets (1/12, 0);
  Q at the root: check 1/6 (3/4 - 5/4) = -1/12, bet 1/6 (3/2 - 1/2) = 1/6,
                 regrets (0, 1/8); Q facing check-bet: regrets (0, 1/12);
  K at the root: check 2/6 3/4 = 1/4, bet 2/6 3/2 = 1/2, regrets (0, 1/8);
  K facing check-bet: fold -1/6, call +1/3, regrets (0, 1/4).
So player 1 bets with every card after iteration 1.  Player 2 then updates
against that strategy (alternation): facing a bet J folds (regrets 1/6, 0),
Q and K call (regrets (0, 1/6) and (0, 1/2)); after a check (now never
reached) every regret is 0 and play stays uniform.
Averages after two iterations, RM+ (weights 1, 2): player 1 bets with
(1/2 + 2)/3 = 5/6 at the root; player 2 folds J / calls Q and K facing a bet
with probability 5/6.  DCFR (weights 1, 4): 0.9 in the same places.
"""
import itertools
from collections import defaultdict

import numpy as np
import pytest

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import synth

EPS = 2.0 ** -40          # the regret-matching noise floor (V = 1 for Kuhn poker)
CARDS = (0, 1, 2)
ACTIONS = {"": "cb", "cb": "fk", "c": "cb", "b": "fk"}     # history -> actions
P1_SETS, P2_SETS = ("", "cb"), ("c", "b")


def _payoff1(c1, c2, h):
    win = 1 if c1 > c2 else -1
    return {"cc": win, "cbf": -1, "cbk": 2 * win, "bf": 1, "bk": 2 * win}[h]


def _actor(h):
    return 0 if h in ("", "cb") else 1


def _cfv(player, s1, s2):
    """Counterfactual value of every (card, history, action) of `player`."""
    out = defaultdict(float)

    def walk(c1, c2, h, reach_opp):
        if h not in ACTIONS:
            u = _payoff1(c1, c2, h)
            return u if player == 0 else -u
        actor = _actor(h)
        card = c1 if actor == 0 else c2
        sig = (s1 if actor == 0 else s2)[(card, h)]
        if actor == player:
            v = 0.0
            for a in ACTIONS[h]:
                va = walk(c1, c2, h + a, reach_opp)
                out[(card, h, a)] += reach_opp / 6.0 * va
                v += sig[a] * va
            return v
        return sum(sig[a] * walk(c1, c2, h + a, reach_opp * sig[a]) for a in ACTIONS[h])

    for c1, c2 in itertools.permutations(CARDS, 2):
        walk(c1, c2, "", 1.0)
    return out


def _uniform(sets):
    return {(c, h): {a: 0.5 for a in ACTIONS[h]} for c in CARDS for h in sets}


def _match(R, sets, positive_part):
    s = {}
    for c in CARDS:
        for h in sets:
            r = {a: (max(R[(c, h, a)], 0.0) if positive_part else R[(c, h, a)]) for a in ACTIONS[h]}
            tot = sum(r.values())
            s[(c, h)] = {a: (r[a] / tot if tot > EPS else 0.5) for a in ACTIONS[h]}
    return s


def _seq(sig, sets):
    """Sequence-form weights of every (card, history, action)."""
    x = {}
    for c in CARDS:
        for h in sets:
            own = 1.0 if h in ("", "c", "b") else sig[(c, "")]["c"]   # player 1 reaches "cb" by checking
            for a in ACTIONS[h]:
                x[(c, h, a)] = own * sig[(c, h)][a]
    return x


def _update(R, cfv, sig, sets, t, dcfr, ab=(1.5, 0.0)):
    for c in CARDS:
        for h in sets:
            v = sum(sig[(c, h)][a] * cfv[(c, h, a)] for a in ACTIONS[h])
            for a in ACTIONS[h]:
                r = R[(c, h, a)] + cfv[(c, h, a)] - v
                if dcfr:
                    ta, tb = t ** ab[0], t ** ab[1]
                    R[(c, h, a)] = r * (ta / (ta + 1.0) if r > 0 else tb / (tb + 1.0))
                else:
                    R[(c, h, a)] = max(r, 0.0)


def _walk_solver(iters, dcfr, ab=(1.5, 0.0), shift=0):
    """Returns per iteration t the averages after t iterations (behavioural,
    {(card, history): {action: p}}) and the regrets after iteration 1.  ab:
    DCFR's discount exponents; shift: discount with t - shift (slips)."""
    s1, s2 = _uniform(P1_SETS), _uniform(P2_SETS)
    R1, R2 = defaultdict(float), defaultdict(float)
    xs, ys = defaultdict(float), defaultdict(float)
    out, first = [], None
    for t in range(1, iters + 1):
        w = float(t) ** 2 if dcfr else float(t)
        for k, v in _seq(s1, P1_SETS).items():
            xs[k] += w * v
        _update(R1, _cfv(0, s1, s2), s1, P1_SETS, max(t - shift, 1), dcfr, ab)
        s1 = _match(R1, P1_SETS, dcfr)
        for k, v in _seq(s2, P2_SETS).items():
            ys[k] += w * v
        _update(R2, _cfv(1, s1, s2), s2, P2_SETS, max(t - shift, 1), dcfr, ab)
        s2 = _match(R2, P2_SETS, dcfr)
        if t == 1:
            first = (dict(R1), dict(R2))
        avg = {}
        for sums, sets in ((xs, P1_SETS), (ys, P2_SETS)):
            for c in CARDS:
                for h in sets:
                    den = sum(sums[(c, h, a)] for a in ACTIONS[h])
                    avg[(c, h)] = {a: (sums[(c, h, a)] / den if den > 0 else 0.5) for a in ACTIONS[h]}
        out.append(avg)
    return out, first


def _oracle_layout(og):
    """(player, seq) -> (history, action) for Kuhn poker, from the oracle's
    sequence table: node 0 / 1 and the action codes (0 fold, 1 check or
    call, 2 bet)."""
    hist = {0: {0: "", 1: "cb"}, 1: {0: "c", 1: "b"}}
    letter = {"": {1: "c", 2: "b"}, "cb": {0: "f", 1: "k"}, "c": {1: "c", 2: "b"}, "b": {0: "f", 1: "k"}}
    out = {}
    for p in (0, 1):
        sq = og.sequences(p)
        for s in range(len(sq["node"])):
            h = hist[p][int(sq["node"][s])]
            out[(p, s)] = (h, letter[h][int(sq["action"][s])])
    return out


def _compare(og, avg_or, avg_walk, p):
    lay = _oracle_layout(og)
    a = avg_or
    for s in range(a.shape[0]):
        h, act = lay[(p, s)]
        for c in CARDS:
            assert abs(a[s, c] - avg_walk[(c, h)][act]) <= 1e-14, (p, s, c, a[s, c], avg_walk[(c, h)][act])


def test_walk_matches_hand_worked_first_iterations():
    for dcfr in (False, True):
        avgs, (R1, R2) = _walk_solver(2, dcfr)
        scale = 0.5 if dcfr else 1.0     # DCFR's first iteration halves every regret
        want1 = {(0, "", "c"): 0.0, (0, "", "b"): 1 / 8, (0, "cb", "f"): 1 / 12, (0, "cb", "k"): 0.0,
                 (1, "", "c"): 0.0, (1, "", "b"): 1 / 8, (1, "cb", "f"): 0.0, (1, "cb", "k"): 1 / 12,
                 (2, "", "c"): 0.0, (2, "", "b"): 1 / 8, (2, "cb", "f"): 0.0, (2, "cb", "k"): 1 / 4}
        for k, v in want1.items():
            got = max(R1[k], 0.0) if dcfr else R1[k]
            assert got == pytest.approx(scale * v, abs=1e-15), k
        want2 = {(0, "b", "f"): 1 / 6, (0, "b", "k"): 0.0, (1, "b", "f"): 0.0, (1, "b", "k"): 1 / 6,
                 (2, "b", "f"): 0.0, (2, "b", "k"): 1 / 2}
        for k, v in want2.items():
            got = max(R2[k], 0.0) if dcfr else R2[k]
            assert got == pytest.approx(scale * v, abs=1e-15), k
        for c in CARDS:
            assert max(R2.get((c, "c", "c"), 0.0), 0.0) == 0.0 and max(R2.get((c, "c", "b"), 0.0), 0.0) == 0.0
        two = avgs[1]
        p = 0.9 if dcfr else 5 / 6
        for c in CARDS:
            assert two[(c, "")]["b"] == pytest.approx(p, abs=1e-15)
            assert two[(c, "c")]["c"] == pytest.approx(0.5, abs=1e-15)
        assert two[(0, "b")]["f"] == pytest.approx(p, abs=1e-15)
        assert two[(1, "b")]["k"] == pytest.approx(p, abs=1e-15)
        assert two[(2, "b")]["k"] == pytest.approx(p, abs=1e-15)


@pytest.mark.parametrize("iters", [1, 2, 3, 4, 5, 6])
def test_oracle_rmplus_schedule(iters):
    og = OracleGame(synth.kuhn_spec())
    _, a1, a2, _ = og.rmplus(iters)
    avgs, _ = _walk_solver(iters, dcfr=False)
    _compare(og, a1, avgs[-1], 0)
    _compare(og, a2, avgs[-1], 1)


@pytest.mark.parametrize("iters", [1, 2, 3, 4, 5, 6])
def test_oracle_dcfr_schedule(iters):
    og = OracleGame(synth.kuhn_spec())
    _, a1, a2, _ = og.dcfr(iters, alpha=1.5, beta=0.0, gamma=2.0)
    avgs, _ = _walk_solver(iters, dcfr=True)
    _compare(og, a1, avgs[-1], 0)
    _compare(og, a2, avgs[-1], 1)


def test_schedule_slips_are_caught():
    """The comparison above would fail for the plausible slips: each altered
    walk differs from the oracle by far more than the tolerance."""
    og = OracleGame(synth.kuhn_spec())
    _, a1, a2, _ = og.rmplus(4)
    lay = _oracle_layout(og)

    def dist(avg):
        d = 0.0
        for (p, s), (h, act) in lay.items():
            arr = a1 if p == 0 else a2
            for c in CARDS:
                d = max(d, abs(arr[s, c] - avg[(c, h)][act]))
        return d

    good, _ = _walk_solver(4, dcfr=False)
    assert dist(good[-1]) <= 1e-14
    # uniform averaging: the averages of the same iterates with weights 1
    s1, s2 = _uniform(P1_SETS), _uniform(P2_SETS)
    R1, R2 = defaultdict(float), defaultdict(float)
    xs, ys = defaultdict(float), defaultdict(float)
    sim_s1, sim_s2 = _uniform(P1_SETS), _uniform(P2_SETS)
    S1, S2 = defaultdict(float), defaultdict(float)
    sx, sy = defaultdict(float), defaultdict(float)
    for t in range(1, 5):
        for k, v in _seq(s1, P1_SETS).items():
            xs[k] += v
        _update(R1, _cfv(0, s1, s2), s1, P1_SETS, t, False)
        s1 = _match(R1, P1_SETS, False)
        for k, v in _seq(s2, P2_SETS).items():
            ys[k] += v
        _update(R2, _cfv(1, s1, s2), s2, P2_SETS, t, False)
        s2 = _match(R2, P2_SETS, False)
        # simultaneous updates: player 2 against the old x
        for k, v in _seq(sim_s1, P1_SETS).items():
            sx[k] += t * v
        for k, v in _seq(sim_s2, P2_SETS).items():
            sy[k] += t * v
        c1, c2 = _cfv(0, sim_s1, sim_s2), _cfv(1, sim_s1, sim_s2)
        _update(S1, c1, sim_s1, P1_SETS, t, False)
        _update(S2, c2, sim_s2, P2_SETS, t, False)
        sim_s1, sim_s2 = _match(S1, P1_SETS, False), _match(S2, P2_SETS, False)

    def beh(xsum, ysum):
        avg = {}
        for sums, sets in ((xsum, P1_SETS), (ysum, P2_SETS)):
            for c in CARDS:
                for h in sets:
                    den = sum(sums[(c, h, a)] for a in ACTIONS[h])
                    avg[(c, h)] = {a: (sums[(c, h, a)] / den if den > 0 else 0.5) for a in ACTIONS[h]}
        return avg

    assert dist(beh(xs, ys)) > 1e-3
    assert dist(beh(sx, sy)) > 1e-3
    # DCFR: swapped discount exponents, or discounts taken at t - 1
    _, d1, d2, _ = og.dcfr(6, alpha=1.5, beta=0.0, gamma=2.0)
    a1, a2 = a1.copy(), a2.copy()
    a1[:], a2[:] = d1, d2
    good, _ = _walk_solver(6, dcfr=True)
    assert dist(good[-1]) <= 1e-14
    swapped, _ = _walk_solver(6, dcfr=True, ab=(0.0, 1.5))
    assert dist(swapped[-1]) > 1e-6
    late, _ = _walk_solver(6, dcfr=True, shift=1)
    assert dist(late[-1]) > 1e-6


@pytest.mark.parametrize("name,spec", [
    ("kuhn", synth.kuhn_spec()),
    ("tiny", synth.tiny_spec()),
    ("micro15_s3", synth.micro_spec(seed=3)),
    ("micro15_s11", synth.micro_spec(seed=11)),
    ("micro15_s29", synth.micro_spec(seed=29)),
])
def test_regret_floor_only_removes_rounding_noise(name, spec):
    """The oracle forms counterfactual values by direct sums over hand pairs,
    so a value that should be zero is exactly zero there, and the floor of
    2^-40 V (reading R17: regret matching plays uniformly at regret sums up
    to it) changes nothing: with the floor and with textbook RM+ (floor 0)
    the averages after 300 iterations are identical bit for bit.  The floor
    matters only for the GPU's Kronecker form, which subtracts card-overlap
    masses and leaves noise of about 1e-17 in place of such zeros."""
    og = OracleGame(spec)
    e0, x0, y0 = og.rmplus_eps(300, 0.0)
    e1, x1, y1 = og.rmplus_eps(300, EPS)
    assert np.array_equal(x0, x1) and np.array_equal(y0, y1) and e0 == e1
    e2, x2, y2, _ = og.rmplus(300)
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2) and e1 == e2
