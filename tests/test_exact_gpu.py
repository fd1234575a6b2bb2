"""Bit-exact products on exact-arithmetic inputs, and the FP64 solver iterate
by iterate on the tiny Kronecker game.

Exact arithmetic: with beliefs whose compatible-pair mass beta is a power of
4, lambda = mu / sqrt(beta) is dyadic; with integer payoffs and small-integer
input vectors every term of every product is a dyadic rational with a few
significant bits, so FP32 and FP64 results are exact and every kernel path
must equal the oracle bit for bit.
  * Kuhn poker with mu = (1, 2, 2) for both players: beta = 5^2 - 9 = 16.
  * a two-card micro game with beliefs in {1, 2}: the first seed whose beta
    (computed by the oracle) is a power of 4.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import kps, synth
from tests.gpu_util import from_library, library_order, to_library

pytestmark = pytest.mark.gpu


def _power_of_4(x):
    if x <= 0:
        return False
    k = round(math.log(x, 4))
    return x == 4.0 ** k


def _kuhn_exact():
    spec = dict(synth.kuhn_spec(), mu1=[1.0, 2.0, 2.0], mu2=[1.0, 2.0, 2.0])
    assert OracleGame(spec).beta == 16.0
    return spec


def _micro_exact():
    for seed in range(2000):
        base = synth.micro_spec(seed=seed, ranks=4, suits=2, nboard=2, beliefs=False)
        r = np.random.default_rng(seed)
        H = synth.num_hands(4, 2, 2, 2)
        spec = dict(base, mu1=r.choice([1.0, 2.0], size=H).tolist(), mu2=r.choice([1.0, 2.0], size=H).tolist())
        if _power_of_4(OracleGame(spec).beta):
            return spec
    raise AssertionError("no exact micro game in 2000 seeds")


EXACT = [("kuhn", _kuhn_exact), ("micro", _micro_exact)]
TDT = {kps.F32: torch.float32, kps.F64: torch.float64}


@pytest.mark.parametrize("kernel", ["tma", "tmem", "vec", "fast"])
@pytest.mark.parametrize("dt", [kps.F32, kps.F64])
@pytest.mark.parametrize("name,mk", EXACT, ids=[e[0] for e in EXACT])
def test_products_bit_exact(name, mk, dt, kernel, monkeypatch):
    if kernel in ("tmem", "tma") and dt == kps.F64:
        pytest.skip("tensor-memory paths are FP32 arithmetic")
    monkeypatch.setenv("KPS_KERNEL", kernel)
    spec = mk()
    og, g = OracleGame(spec), kps.Game(spec)
    order = library_order(spec["strength"])
    inf = g.info()
    for transpose in (False, True):
        n_in = inf["n1"] if transpose else inf["n2"]
        n_out = inf["n2"] if transpose else inf["n1"]
        v = synth.integer_vectors(n_in, og.H, 5, seed=7 + transpose)
        vin = torch.from_numpy(to_library(v, order, inf["hs"])).to("cuda", TDT[dt]).contiguous()
        out = torch.full((5, n_out, inf["hs"]), float("nan"), device="cuda", dtype=TDT[dt])
        (kps.matvec_AT if transpose else kps.matvec_A)(g, vin, out, 5, dtype=dt)
        torch.cuda.synchronize()
        got = from_library(out.double().cpu().numpy(), order, inf["H"])
        want = og.matvec_AT(v) if transpose else og.matvec_A(v)
        assert np.array_equal(got, want), (name, dt, kernel, transpose)


@pytest.mark.parametrize("dt", [kps.F32, kps.F64])
def test_batched_products_bit_exact(dt):
    specs = [_kuhn_exact(), _micro_exact()]
    # a batch needs one hand size per launch: run each game in its own batch and both
    # micro copies together
    for group in ([specs[0]], [specs[1], specs[1]]):
        games = [kps.Game(s) for s in group]
        b = kps.Batch(games)
        ogs = [OracleGame(s) for s in group]
        orders = [library_order(s["strength"]) for s in group]
        off = [b.offsets(p) for p in (0, 1)]
        y = np.zeros(off[1][-1])
        ys = []
        for i, g in enumerate(games):
            inf = g.info()
            v = synth.integer_vectors(inf["n2"], inf["H"], 1, seed=11 + i)[0]
            ys.append(v)
            y[off[1][i]:off[1][i + 1]] = to_library(v, orders[i], inf["hs"]).reshape(-1)
        out = torch.zeros(int(off[0][-1]), dtype=TDT[dt], device="cuda")
        b.matvec_A(torch.from_numpy(y).to("cuda", TDT[dt]), out, dtype=dt)
        torch.cuda.synchronize()
        o = out.double().cpu().numpy()
        for i, g in enumerate(games):
            inf = g.info()
            got = from_library(o[off[0][i]:off[0][i + 1]].reshape(inf["n1"], inf["hs"]), orders[i], inf["H"])
            assert np.array_equal(got, ogs[i].matvec_A(ys[i][None])[0])


def test_fp64_solver_iterate_by_iterate_on_tiny_game():
    """Config 1 (the tiny game, FP64): the average strategies after every
    one of the first 20 iterations equal the oracle's to 1e-12."""
    spec = synth.tiny_spec()
    og = OracleGame(spec)
    g = kps.Game(spec)
    b = kps.Batch([g])
    s = kps.Solver(b, kps.F64)
    order = library_order(spec["strength"])
    inf = g.info()
    x = torch.zeros(int(b.offsets(0)[-1]), dtype=torch.float64, device="cuda")
    y = torch.zeros(int(b.offsets(1)[-1]), dtype=torch.float64, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    for t in range(1, 21):
        s.step(1)
        s.average(x, y, behavioural=True)
        s.exploitability(e)
        torch.cuda.synchronize()
        e_or, a1, a2, _ = og.rmplus(t)
        ax = from_library(x.cpu().numpy().reshape(-1, inf["hs"]), order, inf["H"])
        ay = from_library(y.cpu().numpy().reshape(-1, inf["hs"]), order, inf["H"])
        assert np.max(np.abs(ax - a1)) <= 1e-12 and np.max(np.abs(ay - a2)) <= 1e-12, t
        assert abs(float(e.item()) - e_or) <= 1e-12, t
