"""The TMA-staged FP32 kernel (the default FP32 path) against the FP64 oracle.

Besides the parity checks of test_matvec_gpu.py (which run through this
kernel by default), these cases target what is specific to it:
  - bit-exact products on 1081-hand river games whose beliefs make
    lambda = mu / sqrt(beta) dyadic (beta = 2^20), so that with small-integer
    vectors every FP32 sum is exact: chunks of 17 boxes (16 in tensor memory,
    the 17th in shared memory), the per-card tables and the combination of
    the four chunks are checked bit for bit;
  - the same with every hand in a tie group of 1 to 4 hands (the largest this
    kernel takes), so that the tie corrections run everywhere, across box
    boundaries included;
  - ragged batches (the last CTA's vectors past the batch are zero-filled by
    the copies and clipped on the way out) and batches of one vector;
  - the kernel actually ran (kps_game_kernel).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import kps, synth
from tests.dyadic import dyadic_river
from tests.gpu_util import from_library, library_order, normwise_error, to_library

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ties", [False, True], ids=["river", "river_ties4"])
def test_river_bit_exact(ties):
    spec = dyadic_river(seed=2, ties=ties)
    og, g = OracleGame(spec), kps.Game(spec)
    assert og.beta == float(1 << 20)
    order = library_order(spec["strength"])
    inf = g.info()
    if ties:
        assert inf["max_tie"] == 4
    for transpose in (False, True):
        n_in = inf["n1"] if transpose else inf["n2"]
        n_out = inf["n2"] if transpose else inf["n1"]
        B = 5
        v = synth.integer_vectors(n_in, og.H, B, seed=11 + transpose)
        vin = torch.from_numpy(to_library(v, order, inf["hs"])).to("cuda", torch.float32).contiguous()
        out = torch.full((B, n_out, inf["hs"]), float("nan"), device="cuda")
        (kps.matvec_AT if transpose else kps.matvec_A)(g, vin, out, B)
        torch.cuda.synchronize()
        assert g.kernel(int(transpose)) == "tma"
        o = out.double().cpu().numpy()
        assert np.all(o[..., inf["H"]:] == 0)
        got = from_library(o, order, inf["H"])
        want = og.matvec_AT(v) if transpose else og.matvec_A(v)
        assert np.array_equal(got, want), (ties, transpose, float(np.max(np.abs(got - want))))


@pytest.fixture(scope="module")
def river():
    spec = synth.river_spec(seed=2)
    return spec, OracleGame(spec), kps.Game(spec), library_order(spec["strength"])


@pytest.mark.parametrize("batch", [1, 31, 33, 64])
@pytest.mark.parametrize("transpose", [False, True])
def test_river_batches(river, batch, transpose):
    spec, og, g, order = river
    inf = g.info()
    p = 0 if transpose else 1
    v = synth.simplex_vectors(og.sequences(p)["nact"], og.H, batch, seed=71 + batch)
    n_out = inf["n2"] if transpose else inf["n1"]
    vin = torch.from_numpy(to_library(v, order, inf["hs"])).to("cuda", torch.float32).contiguous()
    out = torch.full((batch, n_out, inf["hs"]), float("nan"), device="cuda")
    (kps.matvec_AT if transpose else kps.matvec_A)(g, vin, out, batch)
    torch.cuda.synchronize()
    assert g.kernel(int(transpose)) == "tma"
    o = out.double().cpu().numpy()
    assert np.all(o[..., inf["H"]:] == 0)
    want = og.matvec_AT(v) if transpose else og.matvec_A(v)
    assert normwise_error(from_library(o, order, inf["H"]), want) <= 1e-5


def test_tie_groups_over_four_fall_back(river):
    """A game with a tie group of 5 hands takes another kernel (same results)."""
    spec = synth.river_spec(seed=2)
    s = np.asarray(spec["strength"])
    order = np.lexsort((np.arange(len(s)), s))
    s = s.copy()
    s[order[100:105]] = s[order[100]]
    spec["strength"] = s.tolist()
    og, g = OracleGame(spec), kps.Game(spec)
    inf = g.info()
    lo = library_order(spec["strength"])
    v = synth.simplex_vectors(og.sequences(1)["nact"], og.H, 3, seed=5)
    vin = torch.from_numpy(to_library(v, lo, inf["hs"])).to("cuda", torch.float32).contiguous()
    out = torch.empty((3, inf["n1"], inf["hs"]), device="cuda")
    kps.matvec_A(g, vin, out, 3)
    torch.cuda.synchronize()
    assert g.kernel(0) != "tma"
    got = from_library(out.double().cpu().numpy(), lo, inf["H"])
    assert normwise_error(got, og.matvec_A(v)) <= 1e-5
