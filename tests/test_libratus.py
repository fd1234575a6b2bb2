"""The Libratus betting menus (appendix "Libratus' betting abstraction"):
per-player, per-situation bet fractions, all-in always, no raise cap.

Pins independent of both builders: a small recursive enumerator of the
betting rules written here, and the number of actions at the root read off
the paper's lists.  Library and oracle must agree with them and with each
other (sequences, terminals, Technique B counts)."""
import numpy as np
import pytest

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import kps, synth

SITS = 5


def _enumerate(menu, c0, total):
    """(sequences of P1, of P2, fold terminals, showdown terminals) of the
    skeleton: P1 acts first; facing more chips a player folds, calls or
    raises, else checks or bets; a bet of fraction f first matches and then
    adds f times the pot; amounts at or above the all-in level are the
    all-in, which is always offered; a call, or a check after a check, is a
    showdown."""
    seqs, folds, shows = [0, 0], [0], [0]

    def node(me, c, naggr, after_check):
        opp = 1 - me
        allin = total
        facing = c[me] < c[opp]
        acts = [("f", c[me]), ("c", min(c[opp], total))] if facing else [("c", c[me])]
        if allin > (c[opp] if facing else c[me]):
            sit = (1 if after_check else 0) if naggr == 0 else min(naggr + 1, SITS - 1)
            amts = {min(c[opp] + f * 2 * c[opp] if facing else c[me] + f * (c[me] + c[opp]), allin)
                    for f in menu[me][sit]}
            amts.add(allin)
            acts += [("r", a) for a in sorted(amts)]
        seqs[me] += len(acts)
        for kind, a in acts:
            nc = list(c)
            nc[me] = a
            if kind == "f":
                folds[0] += 1
            elif kind == "c" and (facing or after_check):
                shows[0] += 1
            elif kind == "c":
                node(opp, nc, naggr, True)
            else:
                node(opp, nc, naggr + 1, False)

    node(0, [c0, c0], 0, False)
    return seqs[0], seqs[1], folds[0], shows[0]


CASES = [(ai, pot) for ai in (0, 1) for pot in (1000.0, 2000.0, 5000.0, 12000.0)]


@pytest.mark.parametrize("ai,pot", CASES)
def test_tree_sizes_match_enumeration(ai, pot):
    spec = synth.libratus_spec(seed=3, ai_player=ai, pot=pot, ranks=5, suits=2, nboard=2)
    want = _enumerate(spec["menu"], pot / 2, 20000.0)
    inf = kps.Game(spec).info()
    og = OracleGame(spec)
    assert (inf["n1"], inf["n2"], inf["T_fold"], inf["T_showdown"]) == want
    assert (og.n1, og.n2, og.TF, og.TS) == want


@pytest.mark.parametrize("ai", [0, 1])
def test_root_actions_follow_the_paper_menu(ai):
    """Player 1 opens: check, the opener's first-action bets, all-in.  With
    a pot of 1000 and 19,500 behind no bet reaches the all-in level, so the
    AI opens with 8 actions (6 bets) and the opponent with 5 (3 bets)."""
    spec = synth.libratus_spec(seed=3, ai_player=ai, ranks=5, suits=2, nboard=2)
    seq = kps.Game(spec).sequences(0)
    root = seq["node"] == 0
    assert int(np.sum(root)) == (8 if ai == 0 else 5)
    amounts = np.sort(seq["amount"][root])
    fr = synth.LIBRATUS_AI[0] if ai == 0 else synth.LIBRATUS_OPPONENT[0]
    want = np.array([500.0] + [500.0 + f * 1000.0 for f in fr] + [20000.0])
    assert np.array_equal(amounts, want)


@pytest.mark.parametrize("ai", [0, 1])
def test_structure_and_counts_match_oracle(ai):
    spec = synth.libratus_spec(seed=4, ai_player=ai, ranks=5, suits=2, nboard=2)
    g, og = kps.Game(spec), OracleGame(spec)
    for p in (0, 1):
        a, b = g.sequences(p), og.sequences(p)
        for key in ("node", "parent", "action", "nact", "amount"):
            assert np.array_equal(a[key], b[key]), (p, key)
    ta, tb = g.terminals(), og.terminals()
    for key in ta:
        assert np.array_equal(ta[key], tb[key]), key
    inf = g.info()
    mine = [inf[k] for k in ("nnz_A", "nnz_Ahat", "nnz_U", "nnz_M", "nnz_V",
                             "pp_nnz_Ahat", "pp_nnz_U", "pp_nnz_M", "pp_nnz_V")]
    assert mine == og.technique_b_counts().tolist()


def test_river_size_libratus_game():
    """The 1081-hand river game with the Libratus menus (AI = player 1)."""
    spec = synth.libratus_spec(seed=2)
    inf = kps.Game(spec).info()
    assert (inf["H"], inf["n1"], inf["n2"], inf["T_fold"], inf["T_showdown"]) == \
        (1081,) + _enumerate(spec["menu"], 500.0, 20000.0)


def test_menu_validation():
    spec = synth.libratus_spec(seed=3, ranks=5, suits=2, nboard=2)
    bad = dict(spec, menu=[[[0.5]] * 5, [[0.5, -1.0]] * 5])
    with pytest.raises(kps.KpsError) as ei:
        kps.Game(bad)
    assert ei.value.status == kps.EINVAL
