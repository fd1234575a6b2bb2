"""Technique B's explicit-factor product on the GPU (this library's sparse
kernels and cuSPARSE) against the oracle's A*y: normwise 1e-12 in FP64 and
1e-5 in FP32, on micro games (one-card and two-card hands, all ties with
zero beliefs) and on the 1081-hand river game."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import kps, synth
from tests.gpu_util import from_library, library_order, normwise_error, to_library
from tests.test_tb_factors import _all_ties_zero_beliefs

pytestmark = pytest.mark.gpu

GAMES = [
    ("tiny", synth.tiny_spec),
    ("micro_raises", lambda: synth.micro_spec(seed=8, ranks=5, suits=2, nboard=3, raise_cap=3, stack=12.0)),
    ("all_ties_zero_beliefs", _all_ties_zero_beliefs),
    ("river", lambda: synth.river_spec(seed=2)),
]
TOL = {kps.F64: 1e-12, kps.F32: 1e-5}
TDT = {kps.F64: torch.float64, kps.F32: torch.float32}


@pytest.fixture(scope="module", params=GAMES, ids=[g[0] for g in GAMES])
def game(request):
    spec = request.param[1]()
    og, g = OracleGame(spec), kps.Game(spec)
    return spec, og, g, kps.TechniqueB(g), library_order(spec["strength"])


@pytest.mark.parametrize("backend", [0, 1], ids=["own", "cusparse"])
@pytest.mark.parametrize("dt", [kps.F64, kps.F32], ids=["f64", "f32"])
def test_technique_b_product_matches_oracle(game, backend, dt):
    spec, og, g, tb, order = game
    inf = g.info()
    batch = 3 if inf["H"] > 500 else 9                     # not a multiple of the 8-vector blocks
    v = synth.simplex_vectors(og.sequences(1)["nact"], og.H, batch, seed=31)
    y = torch.from_numpy(to_library(v, order, inf["hs"])).to("cuda", TDT[dt]).contiguous()
    out = torch.full((batch, inf["n1"], inf["hs"]), float("nan"), device="cuda", dtype=TDT[dt])
    tb.matvec(y, out, batch, backend=backend, dtype=dt)
    torch.cuda.synchronize()
    o = out.double().cpu().numpy()
    assert np.all(o[..., inf["H"]:] == 0.0)                # padding rows of the factors are empty
    got = from_library(o, order, inf["H"])
    assert normwise_error(got, og.matvec_A(v)) <= TOL[dt]


def test_backends_agree_with_fused_kernel_on_river():
    """The three routes to A*y (fused kernel, own sparse kernels, cuSPARSE)
    agree on 16 river vectors in FP32 (each within the FP32 bound of the
    others)."""
    spec = synth.river_spec(seed=2)
    g = kps.Game(spec)
    inf = g.info()
    tb = kps.TechniqueB(g)
    y = torch.rand((16, inf["n2"], inf["hs"]), device="cuda")
    y[..., inf["H"]:] = 0
    outs = []
    for route in ("fused", 0, 1):
        o = torch.empty((16, inf["n1"], inf["hs"]), device="cuda")
        if route == "fused":
            kps.matvec_A(g, y, o, 16)
        else:
            tb.matvec(y, o, 16, backend=route)
        outs.append(o.double().cpu().numpy())
    torch.cuda.synchronize()
    for o in outs[1:]:
        assert normwise_error(o, outs[0]) <= 2e-5


def test_bad_arguments():
    tb = kps.TechniqueB(kps.Game(synth.tiny_spec()))
    y = torch.zeros(8, device="cuda", dtype=torch.bfloat16)
    with pytest.raises(kps.KpsError) as ei:
        tb.matvec(y, y, 1, dtype=kps.BF16)
    assert ei.value.status == kps.ENOTSUP
    with pytest.raises(kps.KpsError) as ei:
        tb.matvec(y, y, 1, backend=2, dtype=kps.F32)
    assert ei.value.status == kps.EINVAL
