"""Turn endgames at the C ABI (kps_turn_*) against the turn oracle.

The oracle (oracle/kps_turn_oracle.c) builds the two-round tree itself (turn
round, river card, river round) and is pinned by its brute-force walk and by
its decomposition into river games (tests/test_turn_oracle.py).  The library
builds the same matrix as a batch of river games (the turn round with
showdowns paying nothing, one block per ending and river card), so these
tests check the composition: block order, sequence numbering, the river
card's chance weight folded into lambda, hands holding the river card, and
each block's own hand order (kps_turn_block).

* Micro decks (two-card hands, three suits, one-card hands, uniform
  beliefs): every entry of A y and A^T x in FP64 (normwise 1e-12 per game)
  and FP32 (1e-5), on ragged vectors of Dirichlet strategies.
* BF16 and FP16 storage (2^-8 / 2^-10 of each game's largest output)
  against the oracle on the same rounded inputs.
* Hands that hold the river card get exactly zero in that block.
* The 52-card turn (1128 hands, 48 river cards per ending): sampled entries
  of both products, each computed one by one by the oracle, within the FP32
  bound against the largest output of the entry's game.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import OracleTurn
from paper_2112_03804_gb300 import kps, synth

pytestmark = pytest.mark.gpu

MICRO = [
    ("two_card", lambda: synth.turn_spec(seed=3, ranks=5, suits=2, strength_top=6)),
    ("two_card_3suits", lambda: synth.turn_spec(seed=5, ranks=4, suits=3, strength_top=8,
                                                bet_frac_t=(0.5, 1.0), raise_cap_t=1)),
    ("one_card", lambda: synth.turn_spec(seed=7, ranks=5, suits=2, cards_per_hand=1, strength_top=4)),
    ("uniform_beliefs", lambda: synth.turn_spec(seed=9, ranks=5, suits=2, strength_top=5, beliefs=False)),
]


class Layout:
    """Conversion between the oracle's [sequence][hand] (canonical hands,
    sequences of all games stacked) and the library's flat batch layout
    (game after game, [sequence][hs], each game's own hand order)."""

    def __init__(self, t: kps.Turn):
        inf = t.info()
        self.H, self.hs, self.games = inf["H"], inf["hs"], inf["games"]
        self.off = [t.offsets(p) for p in (0, 1)]
        self.canon = [t.block(i)[2] for i in range(self.games)]
        self.rows = [np.diff(self.off[p]) // self.hs for p in (0, 1)]
        self.start = [np.concatenate([[0], np.cumsum(self.rows[p])]) for p in (0, 1)]

    def to_library(self, v, p):
        flat = np.zeros(int(self.off[p][-1]))
        for i in range(self.games):
            blk = v[self.start[p][i]:self.start[p][i + 1]]
            w = np.zeros((blk.shape[0], self.hs))
            w[:, :self.H] = blk[:, self.canon[i]]
            flat[self.off[p][i]:self.off[p][i + 1]] = w.reshape(-1)
        return flat

    def from_library(self, flat, p):
        out = np.zeros((int(self.start[p][-1]), self.H))
        for i in range(self.games):
            w = flat[self.off[p][i]:self.off[p][i + 1]].reshape(-1, self.hs)
            assert np.all(w[:, self.H:] == 0)
            out[self.start[p][i]:self.start[p][i + 1]][:, self.canon[i]] = w[:, :self.H]
        return out


def _strategies(og, p, seed):
    sq = og.sequences(p)
    n = len(sq["parent"])
    r = np.random.default_rng(seed)
    beh = np.zeros((n, og.H))
    for s0 in np.unique(sq["node"]):
        na = int(sq["nact"][s0])
        beh[s0:s0 + na] = r.dirichlet(np.ones(na), size=og.H).T
    return og.seqform(p, beh)


def _run(t, lay, v, p_in, dt):
    tdt = {kps.F64: torch.float64, kps.F32: torch.float32}[dt]
    vin = torch.from_numpy(lay.to_library(v, p_in)).to("cuda", tdt)
    out = torch.full((int(lay.off[1 - p_in][-1]),), float("nan"), dtype=tdt, device="cuda")
    (t.matvec_A if p_in == 1 else t.matvec_AT)(vin, out, dt)
    torch.cuda.synchronize()
    return lay.from_library(out.double().cpu().numpy(), 1 - p_in)


@pytest.mark.parametrize("name,mk", MICRO, ids=[m[0] for m in MICRO])
def test_micro_turn_products(name, mk):
    spec = mk()
    og, t = OracleTurn(spec), kps.Turn(spec)
    inf = t.info()
    assert (inf["H"], inf["n1"], inf["n2"]) == (og.H, og.n1, og.n2)
    assert (inf["endings"], inf["blocks"]) == (og.endings, og.blocks)
    assert (inf["turn_n1"], inf["turn_n2"]) == (og.nturn1, og.nturn2)
    lay = Layout(t)
    y, x = _strategies(og, 1, 5), _strategies(og, 0, 6)
    want = {1: og.matvec(y[None])[0], 0: og.matvec(x[None], transpose=True)[0]}
    for dt, tol in ((kps.F64, 1e-12), (kps.F32, 1e-5)):
        for p_in, v in ((1, y), (0, x)):
            got = _run(t, lay, v, p_in, dt)
            w = want[p_in]
            p_out = 1 - p_in
            for i in range(lay.games):
                a, b = lay.start[p_out][i], lay.start[p_out][i + 1]
                scale = np.max(np.abs(w[a:b]))
                assert np.max(np.abs(got[a:b] - w[a:b])) <= tol * scale, (name, dt, p_in, i)


def test_hands_holding_the_river_card_get_zero():
    spec = synth.turn_spec(seed=3, ranks=5, suits=2, strength_top=6)
    t = kps.Turn(spec)
    lay = Layout(t)
    og = OracleTurn(spec)
    y = _strategies(og, 1, 8)
    got = _run(t, lay, y, 1, kps.F32)
    board = set(spec["board"])
    left = [c for c in range(spec["ranks"] * spec["suits"]) if c not in board]
    hands = [(a, b) for i, a in enumerate(left) for b in left[i + 1:]]
    for i in range(1, lay.games):
        e, r, _ = t.block(i)
        assert e >= 0 and r in left
        holds = np.array([r in h for h in hands])
        blk = got[lay.start[0][i]:lay.start[0][i + 1]]
        assert np.all(blk[:, holds] == 0)
        assert np.any(blk[:, ~holds] != 0)


@pytest.fixture(scope="module")
def full_turn():
    spec = synth.turn_spec(seed=2)
    t = kps.Turn(spec)
    og = OracleTurn(spec)
    return spec, t, og, Layout(t)


def test_full_turn_sampled_entries(full_turn):
    spec, t, og, lay = full_turn
    inf = t.info()
    assert inf["H"] == 1128 and inf["blocks"] == inf["endings"] * 48
    assert (inf["n1"], inf["n2"]) == (og.n1, og.n2)
    rng = np.random.default_rng(17)
    y, x = _strategies(og, 1, 31), _strategies(og, 0, 32)
    for p_in, v in ((1, y), (0, x)):
        got = _run(t, lay, v, p_in, kps.F32)
        p_out = 1 - p_in
        games = np.concatenate([[0], rng.choice(np.arange(1, lay.games), size=40, replace=False)])
        for i in games:
            a, b = int(lay.start[p_out][i]), int(lay.start[p_out][i + 1])
            s = a + int(rng.integers(b - a))
            h = int(rng.integers(og.H))
            want = og.entries(v[None], [0], [s], [h], transpose=p_in == 0)[0]
            scale = float(np.max(np.abs(got[a:b])))
            assert abs(got[s, h] - want) <= 1e-5 * scale, (p_in, int(i), s, h)


@pytest.mark.parametrize("dt,tol", [(kps.BF16, 2.0 ** -8), (kps.F16, 2.0 ** -10)], ids=["bf16", "f16"])
def test_micro_turn_half_precision(dt, tol):
    """BF16 / FP16 storage (the staged kernel's 16-bit path, FP32
    arithmetic) against the oracle on the same rounded inputs."""
    spec = synth.turn_spec(seed=3, ranks=5, suits=2, strength_top=6)
    og, t = OracleTurn(spec), kps.Turn(spec)
    lay = Layout(t)
    tdt = {kps.BF16: torch.bfloat16, kps.F16: torch.float16}[dt]
    for p_in, v in ((1, _strategies(og, 1, 5)), (0, _strategies(og, 0, 6))):
        vin = torch.from_numpy(lay.to_library(v, p_in)).to("cuda", tdt)
        rounded = lay.from_library(vin.double().cpu().numpy(), p_in)
        out = torch.full((int(lay.off[1 - p_in][-1]),), float("nan"), dtype=tdt, device="cuda")
        (t.matvec_A if p_in == 1 else t.matvec_AT)(vin, out, dt)
        torch.cuda.synchronize()
        got = lay.from_library(out.double().cpu().numpy(), 1 - p_in)
        want = og.matvec(rounded[None], transpose=p_in == 0)[0]
        p_out = 1 - p_in
        for i in range(lay.games):
            a, b = lay.start[p_out][i], lay.start[p_out][i + 1]
            scale = np.max(np.abs(want[a:b]))
            assert np.max(np.abs(got[a:b] - want[a:b])) <= tol * scale, (dt, p_in, i)
