"""Products and the solver on games with the Libratus betting menus (247
sequences per player at the river size) against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import kps, synth
from tests.gpu_util import from_library, library_order, normwise_error, to_library

pytestmark = pytest.mark.gpu

TDT = {kps.F64: torch.float64, kps.F32: torch.float32}
TOL = {kps.F64: 1e-12, kps.F32: 1e-5}


def _products(spec, batch, dt):
    og, g = OracleGame(spec), kps.Game(spec)
    inf = g.info()
    order = library_order(spec["strength"])
    for transpose in (False, True):
        p_in = 0 if transpose else 1
        v = synth.simplex_vectors(og.sequences(p_in)["nact"], og.H, batch, seed=41 + transpose)
        vin = torch.from_numpy(to_library(v, order, inf["hs"])).to("cuda", TDT[dt]).contiguous()
        n_out = inf["n2"] if transpose else inf["n1"]
        out = torch.full((batch, n_out, inf["hs"]), float("nan"), device="cuda", dtype=TDT[dt])
        (kps.matvec_AT if transpose else kps.matvec_A)(g, vin, out, batch, dtype=dt)
        torch.cuda.synchronize()
        got = from_library(out.double().cpu().numpy(), order, inf["H"])
        want = og.matvec_AT(v) if transpose else og.matvec_A(v)
        assert normwise_error(got, want) <= TOL[dt], (transpose, dt)


@pytest.mark.parametrize("dt", [kps.F64, kps.F32], ids=["f64", "f32"])
@pytest.mark.parametrize("ai", [0, 1])
def test_products_small_deck(ai, dt):
    _products(synth.libratus_spec(seed=5, ai_player=ai, ranks=5, suits=2, nboard=2), 5, dt)


def test_products_river_size():
    """1081 hands, 247 + 247 sequences, 329 terminals (FP32, 2 vectors)."""
    _products(synth.libratus_spec(seed=2), 2, kps.F32)


def test_fp64_rmplus_matches_oracle():
    """A 2000-chip pot (154 sequences per player: the solver keeps every
    sequence of a hand in shared memory, at most 227)."""
    spec = synth.libratus_spec(seed=6, pot=2000.0, ranks=5, suits=2, nboard=2)
    og = OracleGame(spec)
    b = kps.Batch([kps.Game(spec)])
    s = kps.Solver(b, kps.F64)
    s.step(30)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.exploitability(e)
    torch.cuda.synchronize()
    e_or = og.rmplus(30)[0]
    assert abs(float(e.item()) - e_or) <= 1e-9 * max(1.0, abs(e_or))


def test_fp64_rmplus_large_tree_matches_oracle():
    """247 sequences per player (1000-chip pot): the solver runs its node
    kernels with 32 hands per block so that every sequence of a hand fits in
    shared memory."""
    spec = synth.libratus_spec(seed=7, ranks=5, suits=2, nboard=2)
    og = OracleGame(spec)
    assert og.n1 == 247
    b = kps.Batch([kps.Game(spec)])
    s = kps.Solver(b, kps.F64)
    s.step(30)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.exploitability(e)
    torch.cuda.synchronize()
    e_or = og.rmplus(30)[0]
    assert abs(float(e.item()) - e_or) <= 1e-9 * max(1.0, abs(e_or))
