"""Host-side checks of the C ABI (no GPU needed): the library loads and
exports every symbol that include/kps.h declares, and its game builder
produces exactly the oracle's integer structure (sequences, terminals,
hands) and Technique B counts, bit for bit."""
import os
import re

import numpy as np
import pytest

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import kps, synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "kps.h")


def _declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*\s*|kps_status\s+)(kps_\w+)\s*\(", txt, re.M)))


def test_header_declarations_exported():
    syms = _declared_symbols()
    assert "kps_matvec_A" in syms and "kps_sparsify" in syms and len(syms) >= 12
    L = kps.lib()
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(kps.EXPORTED) == syms
    assert "sm_103a" in kps.version()


def _library_order(strength):
    """Ascending strength, ties by canonical index (the ABI contract)."""
    s = np.asarray(strength)
    return np.lexsort((np.arange(len(s)), s))


SPECS = [
    ("tiny", synth.tiny_spec()),
    ("kuhn", synth.kuhn_spec()),
    ("micro2", synth.micro_spec(seed=13, ranks=4, suits=2, nboard=2, cards_per_hand=2)),
    ("micro_nocap", synth.micro_spec(seed=3, ranks=4, suits=2, nboard=1, raise_cap=-1, stack=20.0)),
    ("fig1", dict(ranks=4, suits=2, cards_per_hand=1, board=[], strength=list(range(8)),
                  **synth.fig1_betting())),
    ("river", synth.river_spec(seed=2)),
]


@pytest.mark.parametrize("name,spec", SPECS, ids=[s[0] for s in SPECS])
def test_structure_matches_oracle(name, spec):
    g = kps.Game(spec)
    o = OracleGame(spec)
    inf = g.info()
    assert (inf["H"], inf["n1"], inf["n2"], inf["T"], inf["T_fold"], inf["T_showdown"]) == \
           (o.H, o.n1, o.n2, o.T, o.TF, o.TS)
    assert inf["hs"] % 8 == 0 and inf["hs"] >= inf["H"]
    assert inf["beta"] == pytest.approx(o.beta, rel=1e-12)
    for p in (0, 1):
        a, b = g.sequences(p), o.sequences(p)
        for key in ("node", "parent", "action", "nact"):
            assert np.array_equal(a[key], b[key]), (p, key)
        assert np.array_equal(a["amount"], b["amount"])
    ta, tb = g.terminals(), o.terminals()
    for key in ta:
        assert np.array_equal(ta[key], tb[key]), key
    cards, canon = g.hands()
    assert np.array_equal(canon, _library_order(spec["strength"]))
    assert np.array_equal(cards, o.hands()[canon])


@pytest.mark.parametrize("name,spec", SPECS, ids=[s[0] for s in SPECS])
def test_technique_b_counts_match_oracle(name, spec):
    g = kps.Game(spec)
    inf = g.info()
    mine = [inf[k] for k in ("nnz_A", "nnz_Ahat", "nnz_U", "nnz_M", "nnz_V",
                             "pp_nnz_Ahat", "pp_nnz_U", "pp_nnz_M", "pp_nnz_V")]
    assert mine == OracleGame(spec).technique_b_counts().tolist()


def test_counts_with_zero_beliefs_and_long_ties():
    spec = synth.micro_spec(seed=7, ranks=5, suits=2, nboard=2)
    spec["mu1"] = np.where(np.arange(len(spec["strength"])) % 5 == 0, 0.0, 1.0)
    spec["strength"] = [3] * len(spec["strength"])        # every hand ties
    g = kps.Game(spec)
    inf = g.info()
    assert inf["max_tie"] == inf["H"]
    err, dense = OracleGame(spec).technique_b()
    assert err < 1e-12
    mine = [inf[k] for k in ("nnz_A", "nnz_Ahat", "nnz_U", "nnz_M", "nnz_V",
                             "pp_nnz_Ahat", "pp_nnz_U", "pp_nnz_M", "pp_nnz_V")]
    assert mine == dense.tolist()


def test_fig1_through_the_library():
    spec = dict(ranks=4, suits=2, cards_per_hand=1, board=[], strength=list(range(8)),
                **synth.fig1_betting())
    g = kps.Game(spec)
    inf = g.info()
    assert (inf["T"], inf["T_fold"], inf["T_showdown"], inf["n1"], inf["n2"]) == (21, 10, 11, 16, 16)
    tr = g.terminals()
    assert sorted(set(tr["c1"]) | set(tr["c2"])) == [1875.0, 4687.5, 11718.75, 20000.0]


BAD = [
    dict(cards_per_hand=3),
    dict(board=[0, 0]),
    dict(board=[99]),
    dict(contrib0=[0.0, 1.0]),
    dict(bet_frac=[-0.5]),
    dict(stack=[float("nan"), 1.0]),
]


@pytest.mark.parametrize("patch", BAD)
def test_invalid_specs_rejected(patch):
    spec = synth.tiny_spec()
    spec.update(patch)
    with pytest.raises(kps.KpsError) as ei:
        kps.Game(spec)
    assert ei.value.status == kps.EINVAL


def test_unsupported_deck():
    spec = synth.tiny_spec()
    spec.update(ranks=13, suits=5, strength=list(range(65)))
    with pytest.raises(kps.KpsError) as ei:
        kps.Game(spec)
    assert ei.value.status == kps.ENOTSUP


def test_matvec_argument_errors_without_gpu():
    g = kps.Game(synth.tiny_spec())
    with pytest.raises(kps.KpsError) as ei:
        kps.matvec_A(g, 0, 0, 4, dtype=kps.F32)
    assert ei.value.status == kps.EINVAL
    with pytest.raises(kps.KpsError):
        kps.matvec_A(g, 16, 32, -1, dtype=kps.F32)
    kps.matvec_A(g, 16, 32, 0, dtype=kps.F32)   # batch 0 is a no-op
