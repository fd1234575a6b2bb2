"""The batched RM+ solver and FP64 exploitability against the oracle.

* FP64 storage: after a number of alternating RM+ iterations the average
  behavioural strategies and the exploitability equal the oracle's RM+
  (same update, same averaging) up to rounding: 1e-9.
* Exploitability alone: for random behavioural strategies (no iteration)
  the FP64 best responses equal the oracle's within 1e-12 relative.
* Mixed precision (FP32 / BF16 / FP16 storage of strategies and values,
  FP32 regrets and arithmetic, FP64 exploitability): the tiny Kronecker
  game reaches exploitability below 1e-3 of the pot, and its error against
  the FP64 oracle run is reported and bounded.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import kps, synth
from tests.gpu_util import from_library, library_order, to_library

pytestmark = pytest.mark.gpu


def _setup(specs, dt):
    games = [kps.Game(s) for s in specs]
    b = kps.Batch(games)
    s = kps.Solver(b, dt)
    return games, b, s


def _split(b, games, orders, p, flat):
    off = b.offsets(p)
    out = []
    for i, g in enumerate(games):
        inf = g.info()
        n = inf["n1"] if p == 0 else inf["n2"]
        v = flat[off[i]:off[i + 1]].reshape(n, inf["hs"])
        out.append(from_library(v, orders[i], inf["H"]))
    return out


def _expl(s, n):
    e = torch.zeros(n, dtype=torch.float64, device="cuda")
    b1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    b2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.exploitability(e, b1, b2)
    torch.cuda.synchronize()
    return e.cpu().numpy(), b1.cpu().numpy(), b2.cpu().numpy()


def _averages(s, b, games, orders):
    x = torch.zeros(int(b.offsets(0)[-1]), dtype=torch.float64, device="cuda")
    y = torch.zeros(int(b.offsets(1)[-1]), dtype=torch.float64, device="cuda")
    s.average(x, y, behavioural=True)
    torch.cuda.synchronize()
    return (_split(b, games, orders, 0, x.cpu().numpy()), _split(b, games, orders, 1, y.cpu().numpy()))


SOLVER_SPECS = [
    ("tiny", lambda: [synth.tiny_spec()]),
    ("kuhn+micro", lambda: [synth.micro_spec(seed=3, ranks=4, suits=2, nboard=2),
                            synth.micro_spec(seed=8, ranks=5, suits=2, nboard=3, raise_cap=3, stack=12.0)]),
]


@pytest.mark.parametrize("name,mk", SOLVER_SPECS, ids=[c[0] for c in SOLVER_SPECS])
def test_fp64_solver_matches_oracle_rmplus(name, mk):
    specs = mk()
    games, b, s = _setup(specs, kps.F64)
    orders = [library_order(sp["strength"]) for sp in specs]
    iters = 60
    s.step(25)
    s.step(35)          # two graph launches: the iteration count lives on the device
    assert s.iterations() == iters
    e, _, _ = _expl(s, len(specs))
    ax, ay = _averages(s, b, games, orders)
    for i, sp in enumerate(specs):
        og = OracleGame(sp)
        e_or, a1, a2, _ = og.rmplus(iters)
        assert abs(e[i] - e_or) <= 1e-9 * max(1.0, abs(e_or)), (i, e[i], e_or)
        assert np.max(np.abs(ax[i] - a1)) <= 1e-9
        assert np.max(np.abs(ay[i] - a2)) <= 1e-9


def test_warm_start_matches_oracle():
    """reset() with initial behavioural strategies: the first iteration
    plays them (oracle rmplus with beh1, beh2)."""
    spec = synth.micro_spec(seed=3, ranks=4, suits=2, nboard=2)
    og = OracleGame(spec)
    games, b, s = _setup([spec], kps.F64)
    order = library_order(spec["strength"])
    inf = games[0].info()
    beh = [synth.simplex_vectors(og.sequences(p)["nact"], og.H, 1, seed=20 + p)[0] for p in (0, 1)]
    dev = [torch.from_numpy(to_library(beh[p], order, inf["hs"]).reshape(-1)).to("cuda", torch.float32)
           for p in (0, 1)]
    s.reset(dev[0], dev[1])
    s.step(30)
    e, _, _ = _expl(s, 1)
    b32 = [dev[p].cpu().double().numpy().reshape(-1, inf["hs"]) for p in (0, 1)]
    b32 = [from_library(b32[p], order, inf["H"]) for p in (0, 1)]
    e_or, a1, a2, _ = og.rmplus(30, b32[0], b32[1])
    assert abs(e[0] - e_or) <= 1e-9 * max(1.0, abs(e_or))
    ax, ay = _averages(s, b, games, [order])
    assert np.max(np.abs(ax[0] - a1)) <= 1e-9 and np.max(np.abs(ay[0] - a2)) <= 1e-9


def test_exploitability_of_random_strategies():
    specs = synth.batch_specs(seed=21, n=3) + [synth.micro_spec(seed=4, ranks=4, suits=2, nboard=2)]
    games, b, s = _setup(specs, kps.F32)
    orders = [library_order(sp["strength"]) for sp in specs]
    beh = {0: [], 1: []}
    flat = {}
    for p in (0, 1):
        off = b.offsets(p)
        f = np.zeros(off[-1], dtype=np.float32)
        for i, sp in enumerate(specs):
            og_n = games[i].sequences(p)["nact"]
            H = games[i].info()["H"]
            v = synth.simplex_vectors(og_n, H, 1, seed=50 + 7 * i + p)[0].astype(np.float32)
            beh[p].append(v.astype(np.float64))
            f[off[i]:off[i + 1]] = to_library(v, orders[i], games[i].info()["hs"]).reshape(-1)
        flat[p] = torch.from_numpy(f).cuda()
    s.reset(flat[0], flat[1])          # no iteration: the averages are these strategies
    e, br1, br2 = _expl(s, len(specs))
    for i, sp in enumerate(specs):
        og = OracleGame(sp)
        x, y = og.seqform(0, beh[0][i]), og.seqform(1, beh[1][i])
        e_or, b1_or, b2_or = og.exploitability(x, y)
        # FP32 storage of the strategies: their sequence form is exact in
        # FP64 from the FP32 behavioural inputs up to FP32 rounding of x
        assert abs(br1[i] - b1_or) <= 1e-6 * max(1.0, abs(b1_or)), (i, br1[i], b1_or)
        assert abs(br2[i] - b2_or) <= 1e-6 * max(1.0, abs(b2_or)), (i, br2[i], b2_or)
        assert abs(e[i] - e_or) <= 1e-6 * max(1.0, abs(e_or))


def test_exploitability_fp64_exact_path():
    """FP64 storage end to end: best responses within 1e-12 relative."""
    specs = synth.batch_specs(seed=23, n=2)
    games, b, s = _setup(specs, kps.F64)
    orders = [library_order(sp["strength"]) for sp in specs]
    beh = {0: [], 1: []}
    flat = {}
    for p in (0, 1):
        off = b.offsets(p)
        f = np.zeros(off[-1], dtype=np.float32)
        for i, sp in enumerate(specs):
            H = games[i].info()["H"]
            v = synth.simplex_vectors(games[i].sequences(p)["nact"], H, 1, seed=60 + 7 * i + p)[0]
            v = v.astype(np.float32)
            beh[p].append(v.astype(np.float64))
            f[off[i]:off[i + 1]] = to_library(v, orders[i], games[i].info()["hs"]).reshape(-1)
        flat[p] = torch.from_numpy(f).cuda()
    s.reset(flat[0], flat[1])
    e, br1, br2 = _expl(s, len(specs))
    for i, sp in enumerate(specs):
        og = OracleGame(sp)
        e_or, b1_or, b2_or = og.exploitability(og.seqform(0, beh[0][i]), og.seqform(1, beh[1][i]))
        scale = max(abs(b1_or), abs(b2_or), 1e-300)
        assert abs(br1[i] - b1_or) <= 1e-12 * scale and abs(br2[i] - b2_or) <= 1e-12 * scale


@pytest.mark.parametrize("dt", [kps.F32, kps.BF16, kps.F16])
def test_mixed_precision_reaches_1e3_pot(dt):
    """Tiny Kronecker game, storage `dt`: exploitability below 1e-3 of the
    pot, and the distance of the run's exploitability from the FP64
    oracle's stays below the precision's bound after each block."""
    spec = synth.tiny_spec()
    og = OracleGame(spec)
    games, b, s = _setup([spec], dt)
    block, blocks = 50, 20
    trace = []
    for k in range(blocks):
        s.step(block)
        trace.append(_expl(s, 1)[0][0])
    e_or, _, _, tr_or = og.rmplus(block * blocks, trace_every=block)
    ref = tr_or[block - 1::block]
    err = np.abs(np.array(trace) - ref)
    # strategies and values rounded to the storage type each iteration:
    # the exploitability of the averages differs from the FP64 run by at
    # most a few units of that type's rounding (pot-normalised)
    bound = {kps.F32: 1e-5, kps.BF16: 2.0 ** -6, kps.F16: 2.0 ** -8}[dt]
    assert np.max(err) <= bound, (np.max(err), trace, ref)
    assert min(trace) < 1e-3


@pytest.mark.parametrize("name,mk", SOLVER_SPECS, ids=[c[0] for c in SOLVER_SPECS])
def test_fp64_dcfr_matches_oracle(name, mk):
    """Discounted CFR (alpha 1.5, beta 0, gamma 2) in FP64 storage equals
    the oracle's DCFR: exploitability and sequence-form averages to 1e-9,
    the solver bar (60 iterations of regret dynamics amplify the products'
    rounding differences, ~1e-16, to ~1e-10 here).  With t^2 weights some
    sequences end with a tiny average reach; behavioural strategies there
    are ratios of tiny numbers, so they are compared through the sequence
    form."""
    specs = mk()
    games, b, s = _setup(specs, kps.F64)
    s.set_method(1, 1.5, 0.0, 2.0)
    s.reset()
    orders = [library_order(sp["strength"]) for sp in specs]
    s.step(25)
    s.step(35)
    e, _, _ = _expl(s, len(specs))
    x = torch.zeros(int(b.offsets(0)[-1]), dtype=torch.float64, device="cuda")
    y = torch.zeros(int(b.offsets(1)[-1]), dtype=torch.float64, device="cuda")
    s.average(x, y, behavioural=False)
    torch.cuda.synchronize()
    sx = _split(b, games, orders, 0, x.cpu().numpy())
    sy = _split(b, games, orders, 1, y.cpu().numpy())
    for i, sp in enumerate(specs):
        og = OracleGame(sp)
        e_or, a1, a2, _ = og.dcfr(60, 1.5, 0.0, 2.0)
        assert abs(e[i] - e_or) <= 1e-9 * max(1.0, abs(e_or)), (i, e[i], e_or)
        assert np.max(np.abs(sx[i] - og.seqform(0, a1))) <= 1e-9
        assert np.max(np.abs(sy[i] - og.seqform(1, a2))) <= 1e-9


def test_exploitability_estimate_close_to_fp64():
    """The FP32 estimate used for stopping tests differs from the FP64
    exploitability only by the FP32 rounding of the products: within 1e-5
    of the pot on river games (values are at most a few pots)."""
    specs = [synth.river_spec(seed=sd) for sd in (5, 6, 7)]
    games, b, s = _setup(specs, kps.F32)
    s.step(40)
    e64, _, _ = _expl(s, 3)
    e = torch.zeros(3, dtype=torch.float64, device="cuda")
    s.exploitability_estimate(e)
    torch.cuda.synchronize()
    assert np.max(np.abs(e.cpu().numpy() - e64)) <= 1e-5
    assert np.all(e64 > 0)
