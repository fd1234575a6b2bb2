"""Pins for the FP64 oracle, against facts fixed by the paper and by
mathematics rather than by the oracle itself:

* the terminal table of Fig. 1 and the pot arithmetic of the appendix worked
  example (golden file, transcribed from the paper);
* Kuhn poker's value -1/18 for the first player and its unique equilibrium
  strategy for the second player (closed forms), plus hand-derived entries of
  its payoff matrix and a hand-derived best-response value;
* a brute-force walk of the full game tree (chance deal + skeleton) against
  x^T A y from the explicit matrix, on small random games;
* closed-form card-removal counts for two-card hands from N cards;
* the Technique B identity A = Ahat + U M^-1 V^T (Sec. 4), before and after
  the postprocessing, with the structural nnz counts.
"""
import os

import numpy as np
import pytest

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_skeleton.txt")


def _fig1_game():
    spec = dict(ranks=4, suits=2, cards_per_hand=1, board=[], strength=list(range(8)),
                **synth.fig1_betting())
    return OracleGame(spec)


def _paper_layout(v):
    """[seq][hand] -> the paper's hand-major Kronecker index h*n + s."""
    return np.ascontiguousarray(v.T).reshape(-1)


# ----------------------------------------------------------------- Fig. 1
def test_fig1_terminal_table():
    g = _fig1_game()
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 21
    assert (g.T, g.TF, g.TS) == (21, 10, 11)
    tr = g.terminals()
    seen = set()
    for r in rows:
        label, kind, c1, c2 = r[0], r[-3], float(r[-2]), float(r[-1])
        path = " ".join(r[1:-3])
        t = g.find_terminal(path)
        assert t >= 0, (label, path)
        seen.add(t)
        assert tr["kind"][t] == (0 if kind == "F" else 1), label
        # the figure prints one decimal
        assert abs(tr["c1"][t] - c1) <= 0.05 + 1e-9, (label, tr["c1"][t], c1)
        assert abs(tr["c2"][t] - c2) <= 0.05 + 1e-9, (label, tr["c2"][t], c2)
    assert len(seen) == 21


def test_fig1_sequences_and_worked_example():
    g = _fig1_game()
    # 16 numbered sequences per player in the appendix copy of the figure
    assert (g.n1, g.n2) == (16, 16)
    assert (g.np1, g.np2) == (6, 6)
    tr = g.terminals()
    # node D: the small blind adds 3/4 * (2 * 1875) = 2812.5 on top of 1875
    L = g.find_terminal("b0 f")
    assert tr["c1"][L] == 1875.0 + 2812.5 and tr["c2"][L] == 1875.0
    # T: a raise matches 4687.5 and adds 3/4 of the 9375 pot: 1875+2812.5+7031.25
    T = g.find_terminal("b0 b0 c")
    assert tr["c1"][T] == 1875.0 + 2812.5 + 7031.25 == 11718.75
    # raises that would exceed the stack are the all-in action: no 3/4 raise at K
    assert g.find_terminal("b0 b0 b1 c") == -1


# ------------------------------------------------------------------- Kuhn
def _kuhn():
    return OracleGame(synth.kuhn_spec())


def test_kuhn_payoff_entries_by_hand():
    g = _kuhn()
    assert (g.H, g.n1, g.n2, g.T) == (3, 4, 4, 5)
    assert g.beta == 6.0
    A = g.dense_A()
    n1, n2 = g.n1, g.n2
    J, Q, K = 0, 1, 2
    # P1 sequences: 0 check, 1 bet, 2 fold (after check-bet), 3 call
    # P2 sequences: 0 check, 1 bet (after check), 2 fold, 3 call (facing bet)
    e = lambda h1, s1, h2, s2: A[h1 * n1 + s1, h2 * n2 + s2]
    assert e(K, 1, J, 2) == pytest.approx(1 / 6, abs=1e-15)      # bet, opponent folds
    assert e(J, 1, K, 3) == pytest.approx(-2 / 6, abs=1e-15)     # bet, called, loses 2
    assert e(Q, 0, K, 0) == pytest.approx(-1 / 6, abs=1e-15)     # check-check, loses 1
    assert e(Q, 2, J, 1) == pytest.approx(-1 / 6, abs=1e-15)     # folds to a bet
    assert e(K, 3, Q, 1) == pytest.approx(2 / 6, abs=1e-15)      # calls a bet, wins 2
    for s1 in range(n1):
        for s2 in range(n2):
            assert e(J, s1, J, s2) == 0.0                         # card removal
    assert np.count_nonzero(A) == 6 * 5


def test_kuhn_value_and_equilibrium():
    g = _kuhn()
    expl, avg1, avg2, _ = g.rmplus(4000)
    x, y = g.seqform(0, avg1), g.seqform(1, avg2)
    assert g.value(x, y) == pytest.approx(-1.0 / 18.0, abs=2e-4)
    assert 0.0 <= expl < 2e-4
    J, Q, K = 0, 1, 2
    # second player's unique equilibrium: bluff J with 1/3 after a check,
    # call with Q with 1/3 facing a bet, always bet/call with K
    assert avg2[1, J] == pytest.approx(1 / 3, abs=0.02)
    assert avg2[3, Q] == pytest.approx(1 / 3, abs=0.02)
    assert avg2[1, K] == pytest.approx(1.0, abs=0.02)
    assert avg2[3, K] == pytest.approx(1.0, abs=0.02)
    assert avg2[3, J] == pytest.approx(0.0, abs=0.02)
    assert avg2[1, Q] == pytest.approx(0.0, abs=0.02)


def test_kuhn_best_response_by_hand():
    """Against 'never bet, always call' the first player's best response earns
    (2 + 0 - 1)/3 = 1/3: bet K, anything with Q, check J."""
    g = _kuhn()
    y = np.zeros((4, 3))
    y[0, :] = 1.0   # check after a check
    y[3, :] = 1.0   # call facing a bet
    x = g.seqform(0, np.full((4, 3), 0.5))
    _, br1, br2 = g.exploitability(x, y)
    assert br1 == pytest.approx(1.0 / 3.0, abs=1e-14)
    assert br1 >= g.value(x, y) - 1e-14


# ------------------------------------------------------ brute force vs A
MICRO = [
    dict(seed=11, ranks=5, suits=1, nboard=0, cards_per_hand=1),
    dict(seed=12, ranks=3, suits=2, nboard=0, cards_per_hand=1, beliefs=False),
    dict(seed=13, ranks=4, suits=2, nboard=2, cards_per_hand=2),
    dict(seed=14, ranks=3, suits=3, nboard=1, cards_per_hand=2, bet_frac=(1.0,), raise_cap=3),
    dict(seed=15, ranks=4, suits=2, nboard=1, cards_per_hand=2, ties=False, allow_allin=False),
]


@pytest.mark.parametrize("kw", MICRO)
def test_bruteforce_matches_explicit_matrix(kw):
    g = OracleGame(synth.micro_spec(**kw))
    s1, s2 = g.sequences(0), g.sequences(1)
    b1 = synth.simplex_vectors(s1["nact"], g.H, 1, seed=kw["seed"] + 100)[0]
    b2 = synth.simplex_vectors(s2["nact"], g.H, 1, seed=kw["seed"] + 200)[0]
    x, y = g.seqform(0, b1), g.seqform(1, b2)
    A = g.dense_A()
    lhs = _paper_layout(x) @ A @ _paper_layout(y)
    bf = g.bruteforce_value(b1, b2)
    assert lhs == pytest.approx(bf, rel=1e-12, abs=1e-13)
    # the direct products agree with the explicit matrix and are adjoint
    Ay = g.matvec_A(y)[0]
    assert np.allclose(_paper_layout(Ay), A @ _paper_layout(y), rtol=0, atol=1e-13)
    ATx = g.matvec_AT(x)[0]
    assert np.allclose(_paper_layout(ATx), A.T @ _paper_layout(x), rtol=0, atol=1e-13)
    assert float((x * Ay).sum()) == pytest.approx(float((ATx * y).sum()), rel=1e-12, abs=1e-13)
    # sampled entries
    rng = np.random.default_rng(kw["seed"])
    ss, hh = rng.integers(0, g.n1, 8), rng.integers(0, g.H, 8)
    ent = g.matvec_entries(y[None], np.zeros(8, np.int32), ss, hh)
    assert np.allclose(ent, Ay[ss, hh], rtol=0, atol=1e-14)


def test_zero_sum_and_symmetry_of_card_blocks():
    """Swapping the players' hands in a showdown flips gamma: on a game whose
    two players have identical beliefs, the showdown blocks satisfy
    A_S[h1,h2] = -A_S[h2,h1] (W antisymmetric, Sec. 4)."""
    g = OracleGame(synth.micro_spec(seed=21, ranks=4, suits=2, nboard=2, cards_per_hand=2,
                                    beliefs=False))
    A = g.dense_A()
    tr = g.terminals()
    H, n1, n2 = g.H, g.n1, g.n2
    for t in np.nonzero(tr["kind"] == 1)[0][:3]:
        s1, s2 = tr["s1"][t], tr["s2"][t]
        blk = A[np.arange(H) * n1 + s1][:, np.arange(H) * n2 + s2]
        assert np.allclose(blk, -blk.T, atol=1e-15)


# ------------------------------------------------------ card-removal counts
def test_card_removal_closed_forms():
    """Two-card hands from N=47 cards: each hand is incompatible with
    2(N-1)-1 = 91 hands (itself included) and compatible with C(N-2,2) = 990."""
    spec = synth.river_spec(seed=5)
    spec["strength"] = list(np.random.default_rng(5).permutation(1081))   # no ties
    g = OracleGame(spec)
    cnt = g.technique_b_counts()
    assert g.H == 1081 and g.ncards_left == 47
    assert cnt[1] == 1081 * 91 * g.TF            # nnz(Ahat) = nnz(Hx) * nnz(F)
    assert cnt[0] == 1081 * 990 * g.T            # every compatible pair, every terminal
    assert cnt[2] == 2 * 1081 * g.n1             # U = [Lambda1 (x) I | lambda1 (x) I]
    assert cnt[3] == (2 * 1081 - 1) * g.n1 + g.n1


def test_one_card_closed_forms():
    g = OracleGame(synth.tiny_spec())
    assert (g.H, g.n1, g.n2, g.T, g.TF, g.TS) == (6, 7, 7, 9, 4, 5)
    assert g.beta == 30.0                        # 6 * 5 ordered pairs, mu = 1
    cnt = g.technique_b_counts()
    # 30 compatible pairs on fold terminals, 24 non-tied (3 ranks x 2 suits) on showdowns
    assert cnt[0] == 30 * 4 + 24 * 5 == 240


# --------------------------------------------------------------- Technique B
@pytest.mark.parametrize("kw", MICRO + [dict(seed=31, ranks=4, suits=2, nboard=0, cards_per_hand=2)])
def test_technique_b_identity_and_counts(kw):
    g = OracleGame(synth.micro_spec(**kw))
    err, cnt = g.technique_b()
    assert 0.0 <= err < 1e-12
    assert np.array_equal(cnt, g.technique_b_counts())
    assert cnt[6] <= cnt[2] and cnt[7] <= cnt[3] and cnt[8] == cnt[4]


def test_technique_b_tiny_game_counts():
    g = OracleGame(synth.tiny_spec())
    err, cnt = g.technique_b()
    assert err < 1e-15
    # nnz(A), Ahat, U, M, V before; Ahat, U, M, V after postprocessing
    assert cnt.tolist() == [240, 24, 84, 84, 84, 24, 54, 29, 84]


# ------------------------------------------------------------------- solver
def test_rmplus_tiny_converges():
    g = OracleGame(synth.tiny_spec())
    expl, _, _, tr = g.rmplus(600, trace_every=50)
    pts = tr[49::50]
    assert np.all(pts >= 0)
    assert pts[-1] < pts[0]
    assert expl < 1e-3


def test_synth_simplex_vectors():
    v = synth.simplex_vectors([2, 3, 1], 5, 4, seed=3)
    assert v.shape == (4, 6, 5)
    assert np.allclose(v[:, 0:2].sum(1), 1) and np.allclose(v[:, 2:5].sum(1), 1)
    assert np.allclose(v[:, 5], 1)


def test_regret_floor_kuhn_by_hand():
    """Kuhn poker: the largest contribution at a terminal is 2 (ante plus
    bet), beliefs are 1, each player has 3 hands and 6 compatible deals, so
    V = 2 * 1 * 3 / 6 = 1 for both players."""
    og = OracleGame(synth.kuhn_spec())
    assert og.regret_floor(0, 1.0) == pytest.approx(1.0, rel=1e-15)
    assert og.regret_floor(1, 1.0) == pytest.approx(1.0, rel=1e-15)
    assert og.regret_floor(0, 2.0 ** -40) == pytest.approx(2.0 ** -40, rel=1e-15)


def _kuhn_equilibrium():
    """The equilibrium of Kuhn poker with alpha = 0 (closed form): player 1
    always checks, folds J and calls K facing a bet, calls with Q 1/3;
    player 2 bets K and bluffs J 1/3 after a check, calls K and Q 1/3."""
    b1 = np.array([[1, 1, 1], [0, 0, 0], [1, 2 / 3, 0], [0, 1 / 3, 1]], dtype=float)
    b2 = np.array([[2 / 3, 1, 0], [1 / 3, 0, 1], [1, 2 / 3, 0], [0, 1 / 3, 1]], dtype=float)
    return b1, b2


def test_kuhn_equilibrium_is_a_fixed_point_of_warm_rmplus():
    """Warm start at an equilibrium: regrets kappa V b (regret matching gives
    b back) stay proportional to b because the supported actions are
    indifferent, so the iterates and the average stay at the equilibrium;
    a cold start is far from it after the same iterations.  With kappa = 0
    and a large t0 the average is dominated by the initial strategy."""
    g = _kuhn()
    b1, b2 = _kuhn_equilibrium()
    e0, _, _ = g.exploitability(g.seqform(0, b1), g.seqform(1, b2))
    assert abs(e0) < 1e-14
    e_warm, a1, a2, _ = g.rmplus_warm(10, b1, b2, kappa=1.0, t0=50)
    assert e_warm < 1e-12
    assert np.max(np.abs(a1 - b1)) < 1e-9 and np.max(np.abs(a2 - b2)) < 1e-9
    e_cold, _, _, _ = g.rmplus(10)
    assert e_cold > 1e-2
    e_avg, _, _, _ = g.rmplus_warm(10, b1, b2, kappa=0.0, t0=1_000_000)
    assert e_avg < 1e-3
    # kappa = 0, t0 = 0 is plain RM+ from the given strategy
    e1, c1, c2, _ = g.rmplus_warm(7, b1, b2, kappa=0.0, t0=0)
    e2, d1, d2, _ = g.rmplus(7, b1, b2)
    assert e1 == e2 and np.array_equal(c1, d1) and np.array_equal(c2, d2)


def test_dcfr_two_iterations_equal_rmplus_with_linear_weights():
    """After one iteration DCFR's regrets are (q - v)/2 (both discount
    factors are 1/2 at t = 1), whose positive parts point the same way as
    RM+'s max(0, q - v): the second iteration plays the same strategies, so
    with gamma = 1 the averages after two iterations are RM+'s exactly."""
    for spec in (synth.kuhn_spec(), synth.micro_spec(seed=3, ranks=4, suits=2, nboard=2)):
        g = OracleGame(spec)
        e1, a1, b1, _ = g.dcfr(2, alpha=1.5, beta=0.0, gamma=1.0)
        e2, a2, b2, _ = g.rmplus(2)
        assert np.array_equal(a1, a2) and np.array_equal(b1, b2) and e1 == e2


def test_dcfr_solves_kuhn():
    """Kuhn poker: DCFR(1.5, 0, 2) reaches the closed-form value -1/18 and a
    small exploitability, decreasing along the run."""
    g = _kuhn()
    expl, avg1, avg2, tr = g.dcfr(2000, trace_every=500)
    x, y = g.seqform(0, avg1), g.seqform(1, avg2)
    assert g.value(x, y) == pytest.approx(-1.0 / 18.0, abs=2e-4)
    assert 0.0 <= expl < 2e-4
    pts = tr[499::500]
    assert np.all(np.diff(pts) <= 1e-12)
