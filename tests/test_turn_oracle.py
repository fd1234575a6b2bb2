"""Pins for the turn-endgame oracle (oracle/kps_turn_oracle.c, end of Sec. 3).

* Brute force: a walk of the whole two-round tree (chance deal, turn round,
  river card drawn over the cards in neither hand, river round) gives the
  same expected payoff as x^T A y with the sequence forms of the same
  behavioural strategies, on micro decks with two-card and one-card hands,
  ties and beliefs.
* Block structure: the product equals its parts computed with the RIVER
  oracle (kps_oracle.c, an independent tree builder pinned by Fig. 1, Kuhn
  poker and its own brute force): the turn round's folds (a river game on
  the turn board whose showdowns pay nothing, all strengths equal), and for
  every (ending, river card) a river game on the board plus that card,
  started from the ending's contributions with the chips left behind, its
  hands matched by their cards, scaled by beta_river / (beta_turn (N - 2k)):
  the river block's own chance normalisation replaced by the turn deal's
  times the probability of the river card.
* Adjointness x^T (A y) = (A^T x)^T y.
"""
import numpy as np
import pytest

from oracle.oracle import OracleGame, OracleTurn
from paper_2112_03804_gb300 import synth

SPECS = [
    ("two_card", lambda: synth.turn_spec(seed=3, ranks=5, suits=2, strength_top=6)),
    ("two_card_3suits", lambda: synth.turn_spec(seed=5, ranks=4, suits=3, strength_top=8,
                                                bet_frac_t=(0.5, 1.0), raise_cap_t=1)),
    ("one_card", lambda: synth.turn_spec(seed=7, ranks=5, suits=2, cards_per_hand=1, strength_top=4)),
    ("uniform_beliefs", lambda: synth.turn_spec(seed=9, ranks=5, suits=2, strength_top=5, beliefs=False)),
]


def _behavioural(og, p, seed):
    sq = og.sequences(p)
    n = len(sq["parent"])
    r = np.random.default_rng(seed)
    beh = np.zeros((n, og.H))
    for s0 in np.unique(sq["node"]):
        na = int(sq["nact"][s0])
        beh[s0:s0 + na] = r.dirichlet(np.ones(na), size=og.H).T
    return beh


@pytest.mark.parametrize("name,mk", SPECS, ids=[s[0] for s in SPECS])
def test_bruteforce_equals_bilinear_form(name, mk):
    og = OracleTurn(mk())
    for seed in range(3):
        b1, b2 = _behavioural(og, 0, 10 + seed), _behavioural(og, 1, 20 + seed)
        x, y = og.seqform(0, b1), og.seqform(1, b2)
        v = float(np.sum(x * og.matvec(y[None])[0]))
        assert v == pytest.approx(og.bruteforce_value(b1, b2), rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("name,mk", SPECS, ids=[s[0] for s in SPECS])
def test_adjoint(name, mk):
    og = OracleTurn(mk())
    r = np.random.default_rng(4)
    x = r.normal(size=(2, og.n1, og.H))
    y = r.normal(size=(2, og.n2, og.H))
    lhs = np.einsum("bsh,bsh->b", x, og.matvec(y))
    rhs = np.einsum("bsh,bsh->b", og.matvec(x, transpose=True), y)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def _hands(spec, board):
    left = [c for c in range(spec["ranks"] * spec["suits"]) if c not in set(board)]
    if spec["cards_per_hand"] == 1:
        return [(c,) for c in left]
    return [(a, b) for i, a in enumerate(left) for b in left[i + 1:]]


@pytest.mark.parametrize("name,mk", SPECS, ids=[s[0] for s in SPECS])
def test_blocks_equal_river_games(name, mk):
    spec = mk()
    og = OracleTurn(spec)
    k = spec["cards_per_hand"]
    ncard = spec["ranks"] * spec["suits"]
    turn_hands = _hands(spec, spec["board"])
    H = len(turn_hands)
    mu1 = spec["mu1"] if spec["mu1"] is not None else np.ones(H)
    mu2 = spec["mu2"] if spec["mu2"] is not None else np.ones(H)
    base = dict(ranks=spec["ranks"], suits=spec["suits"], cards_per_hand=k, allow_allin=False)
    # the turn round as a river game with equal strengths: folds only
    turn = OracleGame(dict(base, board=spec["board"], stack=spec["stack"], contrib0=spec["contrib0"],
                           bet_frac=spec["bet_frac_t"], raise_cap=spec["raise_cap_t"],
                           strength=[0] * H, mu1=mu1, mu2=mu2))
    assert turn.beta == pytest.approx(og.beta, rel=1e-14)
    assert (turn.n1, turn.n2) == (og.nturn1, og.nturn2)
    tr = turn.terminals()
    ends = [t for t in range(turn.T) if tr["kind"][t] == 1]
    assert len(ends) == og.endings
    r = np.random.default_rng(1)
    y = r.normal(size=(og.n2, og.H))
    x = r.normal(size=(og.n1, og.H))
    got_A = og.matvec(y[None])[0]
    got_AT = og.matvec(x[None], transpose=True)[0]
    want_A = np.zeros_like(got_A)
    want_AT = np.zeros_like(got_AT)
    want_A[:og.nturn1] = turn.matvec_A(y[None, :og.nturn2])[0]
    want_AT[:og.nturn2] = turn.matvec_AT(x[None, :og.nturn1])[0]
    o1, o2 = og.nturn1, og.nturn2
    for t in ends:
        c = tr["c1"][t]
        assert c == tr["c2"][t]
        stack = [spec["contrib0"][p] + spec["stack"][p] - c for p in (0, 1)]
        for card in range(ncard):
            if card in spec["board"]:
                continue
            board = sorted(spec["board"] + [card])
            rh = _hands(spec, board)
            idx = np.array([turn_hands.index(h) for h in rh])
            rg = OracleGame(dict(base, board=board, stack=stack, contrib0=[c, c], bet_frac=spec["bet_frac_r"],
                                 raise_cap=spec["raise_cap_r"],
                                 strength=[int(spec["strength"][card][i]) for i in idx],
                                 mu1=np.asarray(mu1)[idx], mu2=np.asarray(mu2)[idx]))
            scale = rg.beta / (og.beta * (og.N - 2 * k))
            ya = y[o2:o2 + rg.n2][:, idx]
            xa = x[o1:o1 + rg.n1][:, idx]
            want_A[o1:o1 + rg.n1][:, idx] = scale * rg.matvec_A(ya[None])[0]
            want_AT[o2:o2 + rg.n2][:, idx] = scale * rg.matvec_AT(xa[None])[0]
            o1 += rg.n1
            o2 += rg.n2
    assert (o1, o2) == (og.n1, og.n2)
    scale_A = np.max(np.abs(want_A))
    assert np.max(np.abs(got_A - want_A)) <= 1e-12 * scale_A
    assert np.max(np.abs(got_AT - want_AT)) <= 1e-12 * np.max(np.abs(want_AT))
