"""Technique B's explicit factors (Sec. 4) as built by the library, on the
host: their nonzero counts equal the oracle's Technique B counts (before
postprocessing), and Ahat + U M^-1 V^T rebuilt densely from the exported
CSR equals the oracle's payoff matrix A (the oracle's products applied to
unit vectors), entry by entry."""
import numpy as np
import pytest

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import kps, synth
from tests.gpu_util import library_order

SPECS = [
    ("tiny", synth.tiny_spec()),
    ("kuhn", synth.kuhn_spec()),
    ("micro_two_card", synth.micro_spec(seed=3, ranks=4, suits=2, nboard=2)),
    ("micro_raises", synth.micro_spec(seed=8, ranks=5, suits=2, nboard=3, raise_cap=3, stack=12.0)),
]


def _all_ties_zero_beliefs():
    spec = synth.micro_spec(seed=7, ranks=5, suits=2, nboard=2)
    spec["mu1"] = np.where(np.arange(len(spec["strength"])) % 5 == 0, 0.0, 1.0)
    spec["mu2"] = np.where(np.arange(len(spec["strength"])) % 7 == 3, 0.0, 1.0)
    spec["strength"] = [3] * len(spec["strength"])
    return spec


SPECS.append(("all_ties_zero_beliefs", _all_ties_zero_beliefs()))
SPECS.append(("libratus_menus", synth.libratus_spec(seed=3, pot=5000.0, ranks=4, suits=2, nboard=2)))


def _dense(csr):
    (rows, cols), rowptr, col, val = csr
    d = np.zeros((rows, cols))
    for r in range(rows):
        for k in range(rowptr[r], rowptr[r + 1]):
            d[r, col[k]] += val[k]
    return d


def _oracle_A_library_layout(spec, hs):
    """A in the library's [seq][hs] layout (rows s1*hs + h1, columns
    s2*hs + h2, library hand order) from the oracle's products on unit
    vectors."""
    og = OracleGame(spec)
    H, n1, n2 = og.H, og.n1, og.n2
    order = library_order(spec["strength"])
    E = np.zeros((n2 * H, n2, H))
    for s2 in range(n2):
        for i in range(H):
            E[s2 * H + i, s2, order[i]] = 1.0
    cols = og.matvec_A(E)                        # [n2*H][n1][H] canonical
    A = np.zeros((n1 * hs, n2 * hs))
    for s2 in range(n2):
        for i2 in range(H):
            c = cols[s2 * H + i2]
            for s1 in range(n1):
                A[s1 * hs:s1 * hs + H, s2 * hs + i2] = c[s1, order]
    return A


@pytest.mark.parametrize("name,spec", SPECS, ids=[s[0] for s in SPECS])
def test_factor_sizes_match_oracle_counts(name, spec):
    tb = kps.TechniqueB(kps.Game(spec))
    sz = tb.sizes()
    cnt = OracleGame(spec).technique_b_counts()
    assert [sz["nnz_Ahat"], sz["nnz_U"], sz["nnz_M"], sz["nnz_V"]] == cnt[1:5].tolist()


@pytest.mark.parametrize("name,spec", SPECS, ids=[s[0] for s in SPECS])
def test_factors_rebuild_A(name, spec):
    g = kps.Game(spec)
    hs = g.info()["hs"]
    tb = kps.TechniqueB(g)
    Ahat, U, M, Vt = (_dense(tb.export(w)) for w in (tb.AHAT, tb.U, tb.M, tb.VT))
    sz = tb.sizes()
    assert Ahat.shape == (sz["R"], sz["C"]) and U.shape == (sz["R"], sz["m"])
    assert M.shape == (sz["m"], sz["m"]) and Vt.shape == (sz["m"], sz["C"])
    # M unit lower triangular with at most two nonzeros per row
    assert np.allclose(np.diag(M), 1.0) and not np.any(np.triu(M, 1))
    assert np.all((M != 0).sum(axis=1) <= 2)
    A = Ahat + U @ np.linalg.solve(M, Vt)
    want = _oracle_A_library_layout(spec, hs)
    assert np.max(np.abs(A - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))


def test_river_factor_sizes():
    """The 1081-hand river game: factor sizes equal the oracle's counts."""
    spec = synth.river_spec(seed=2)
    tb = kps.TechniqueB(kps.Game(spec))
    sz = tb.sizes()
    cnt = OracleGame(spec).technique_b_counts()
    assert [sz["nnz_Ahat"], sz["nnz_U"], sz["nnz_M"], sz["nnz_V"]] == cnt[1:5].tolist()
