"""Parity of the CUDA products A*y and A^T*x against the FP64 oracle.

Tolerances (normwise, max|gpu - oracle| / max|oracle|): 1e-12 for FP64,
1e-5 for FP32.  BF16/FP16 storage (FP32 arithmetic) is compared with the
oracle on the same rounded inputs; its bound 2^-8 (BF16) / 2^-10 (FP16)
comes from rounding the output once.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import kps, synth
from tests.gpu_util import from_library, library_order, normwise_error, to_library

pytestmark = pytest.mark.gpu

TOL = {kps.F64: 1e-12, kps.F32: 1e-5, kps.BF16: 2.0 ** -8, kps.F16: 2.0 ** -10}
TDT = {kps.F64: torch.float64, kps.F32: torch.float32, kps.BF16: torch.bfloat16, kps.F16: torch.float16}


def _run(game, order, v_canon, transpose, dt):
    inf = game.info()
    n_out = inf["n2"] if transpose else inf["n1"]
    B = v_canon.shape[0]
    vin = torch.from_numpy(to_library(v_canon, order, inf["hs"])).to("cuda", TDT[dt]).contiguous()
    out = torch.full((B, n_out, inf["hs"]), float("nan"), device="cuda", dtype=TDT[dt])
    (kps.matvec_AT if transpose else kps.matvec_A)(game, vin, out, B, dtype=dt)
    torch.cuda.synchronize()
    o = out.to(torch.float64).cpu().numpy()
    assert np.all(o[..., inf["H"]:] == 0), "padding must be written as zero"
    return from_library(o, order, inf["H"]), vin


def _inputs(og, batch, seed, transpose):
    p = 0 if transpose else 1
    return synth.simplex_vectors(og.sequences(p)["nact"], og.H, batch, seed=seed)


CASES = [
    ("tiny", synth.tiny_spec, 3),
    ("kuhn", synth.kuhn_spec, 2),
    ("micro2", lambda: synth.micro_spec(seed=13, ranks=4, suits=2, nboard=2), 5),
    ("micro_alltie", lambda: dict(synth.micro_spec(seed=9, ranks=5, suits=2, nboard=2),
                                  strength=[7] * 28), 4),
    ("fig1", lambda: dict(ranks=4, suits=2, cards_per_hand=1, board=[],
                          strength=[0, 0, 1, 2, 2, 2, 3, 3], **synth.fig1_betting()), 3),
    ("micro_nocap", lambda: synth.micro_spec(seed=3, ranks=4, suits=2, nboard=1,
                                             raise_cap=-1, stack=20.0), 33),
]


@pytest.mark.parametrize("dt", [kps.F64, kps.F32])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("name,mk,batch", CASES, ids=[c[0] for c in CASES])
def test_small_games_match_oracle(name, mk, batch, transpose, dt):
    spec = mk()
    og, g = OracleGame(spec), kps.Game(spec)
    order = library_order(spec["strength"])
    v = _inputs(og, batch, seed=17, transpose=transpose)
    got, _ = _run(g, order, v, transpose, dt)
    want = og.matvec_AT(v) if transpose else og.matvec_A(v)
    assert normwise_error(got, want) <= TOL[dt]


@pytest.fixture(scope="module")
def river():
    spec = synth.river_spec(seed=2)
    return spec, OracleGame(spec), kps.Game(spec), library_order(spec["strength"])


KERNELS = ["tma", "tmem", "vec", "fast"]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("transpose", [False, True])
def test_river_fp32_ragged_batch(river, transpose, kernel, monkeypatch):
    """1081 hands, 43+43 sequences, 37 vectors: many tiles, a ragged last CTA,
    through each kernel path."""
    monkeypatch.setenv("KPS_KERNEL", kernel)
    spec, og, g, order = river
    v = _inputs(og, 37, seed=23, transpose=transpose)
    got, _ = _run(g, order, v, transpose, kps.F32)
    want = og.matvec_AT(v) if transpose else og.matvec_A(v)
    assert normwise_error(got, want) <= 1e-5


def test_river_fp64(river):
    spec, og, g, order = river
    v = _inputs(og, 3, seed=29, transpose=False)
    got, _ = _run(g, order, v, False, kps.F64)
    assert normwise_error(got, og.matvec_A(v)) <= 1e-12
    x = _inputs(og, 3, seed=31, transpose=True)
    got, _ = _run(g, order, x, True, kps.F64)
    assert normwise_error(got, og.matvec_AT(x)) <= 1e-12


@pytest.mark.parametrize("kernel", ["tmem", "fast"])
@pytest.mark.parametrize("dt", [kps.BF16, kps.F16])
def test_river_half_storage(river, dt, kernel, monkeypatch):
    monkeypatch.setenv("KPS_KERNEL", kernel)
    spec, og, g, order = river
    v = _inputs(og, 5, seed=37, transpose=False)
    rounded = torch.from_numpy(v).to(TDT[dt]).to(torch.float64).numpy()
    got, _ = _run(g, order, rounded, False, dt)
    err = normwise_error(got, og.matvec_A(rounded))
    assert err <= TOL[dt]
    # error of the whole mixed-precision path against unrounded FP64 inputs
    err_total = normwise_error(got, og.matvec_A(v))
    assert err_total <= 4 * TOL[dt]


def test_adjoint_and_determinism(river):
    spec, og, g, order = river
    inf = g.info()
    y = _inputs(og, 4, seed=41, transpose=False)
    x = _inputs(og, 4, seed=43, transpose=True)
    Ay, _ = _run(g, order, y, False, kps.F64)
    ATx, _ = _run(g, order, x, True, kps.F64)
    lhs = np.einsum("bsh,bsh->b", x, Ay)
    rhs = np.einsum("bsh,bsh->b", ATx, y)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-15)
    a1, _ = _run(g, order, y, False, kps.F32)
    a2, _ = _run(g, order, y, False, kps.F32)
    assert np.array_equal(a1, a2)


def test_full_size_sampled_entries(river):
    """The benchmark workload (1024 vectors, FP32) checked on sampled outputs
    that the oracle computes one by one."""
    spec, og, g, order = river
    inf = g.info()
    B = 1024
    y = synth.simplex_vectors(og.sequences(1)["nact"], og.H, B, seed=3, dtype=np.float32)
    yl = torch.from_numpy(to_library(y, order, inf["hs"])).cuda()
    out = torch.empty((B, inf["n1"], inf["hs"]), device="cuda", dtype=torch.float32)
    kps.matvec_A(g, yl, out, B)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    nb = 48
    b = rng.integers(0, B, nb)
    s = rng.integers(0, inf["n1"], nb)
    h = rng.integers(0, inf["H"], nb)
    want = og.matvec_entries(y.astype(np.float64), b, s, h)
    pos = np.argsort(order)          # canonical hand -> library position
    got = out[torch.from_numpy(b), torch.from_numpy(s), torch.from_numpy(pos[h])].double().cpu().numpy()
    scale = float(out.abs().max())
    assert np.max(np.abs(got - want)) / scale <= 1e-5
    assert torch.all(out[..., inf["H"]:] == 0)


def test_host_buffer_variant(river):
    spec, og, g, order = river
    inf = g.info()
    y = _inputs(og, 6, seed=47, transpose=False).astype(np.float32)
    yl = np.ascontiguousarray(to_library(y, order, inf["hs"]))
    out = np.zeros((6, inf["n1"], inf["hs"]), dtype=np.float32)
    kps.matvec_A_host(g, yl, out, 6, kps.F32)
    got = from_library(out, order, inf["H"])
    assert normwise_error(got, og.matvec_A(y.astype(np.float64))) <= 1e-5


def test_host_buffer_chunks_match_device_path(river):
    """37 vectors (eight uneven chunks on the copy/product/copy streams), both
    directions: within the FP32 bound of the oracle, and equal bit for bit
    to the device-resident product launched on the same chunks of vectors
    (the copies neither lose nor reorder data; a single 37-vector launch
    groups columns into tiles differently, and a tile's column kinds select
    the scan variant, so it may differ in the last bit)."""
    spec, og, g, order = river
    inf = g.info()
    batch, nch = 37, 8
    bounds = [batch * c // nch for c in range(nch + 1)]
    for transpose in (False, True):
        n_out = inf["n2"] if transpose else inf["n1"]
        v = _inputs(og, batch, seed=61, transpose=transpose).astype(np.float32)
        vl = np.ascontiguousarray(to_library(v, order, inf["hs"]))
        out = np.zeros((batch, n_out, inf["hs"]), dtype=np.float32)
        (kps.matvec_AT_host if transpose else kps.matvec_A_host)(g, vl, out, batch, kps.F32)
        want = og.matvec_AT(v.astype(np.float64)) if transpose else og.matvec_A(v.astype(np.float64))
        assert normwise_error(from_library(out, order, inf["H"]), want) <= 1e-5
        vd = torch.from_numpy(vl).cuda()
        dev = torch.empty((batch, n_out, inf["hs"]), device="cuda")
        for c in range(nch):
            b0, b1 = bounds[c], bounds[c + 1]
            (kps.matvec_AT if transpose else kps.matvec_A)(g, vd[b0:b1], dev[b0:b1], b1 - b0)
        torch.cuda.synchronize()
        assert np.array_equal(out, dev.cpu().numpy())


def test_overlap_rejected(river):
    spec, og, g, order = river
    inf = g.info()
    buf = torch.zeros(2 * inf["n1"] * inf["hs"], device="cuda")
    with pytest.raises(kps.KpsError) as ei:
        kps.matvec_A(g, buf, buf, 1)
    assert ei.value.status == kps.EINVAL


@pytest.fixture(scope="module")
def river_ties():
    spec = synth.river_spec(seed=6)
    spec["strength"] = [s // 40 for s in spec["strength"]]      # tie groups of up to ~15 hands
    return spec, OracleGame(spec), kps.Game(spec), library_order(spec["strength"])


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("warps", ["1", "3", "4", "6", "8"])
@pytest.mark.parametrize("transpose", [False, True])
def test_river_many_ties_warp_counts(river_ties, warps, transpose, kernel, monkeypatch):
    """Tie groups inside tiles, several hand chunks per CTA, each kernel path
    (FP64 runs on the vectorised or scalar path)."""
    spec, og, g, order = river_ties
    monkeypatch.setenv("KPS_WARPS", warps)
    monkeypatch.setenv("KPS_KERNEL", kernel)
    v = _inputs(og, 5, seed=53, transpose=transpose)
    want = og.matvec_AT(v) if transpose else og.matvec_A(v)
    got, _ = _run(g, order, v, transpose, kps.F64)
    assert normwise_error(got, want) <= 1e-12
    got, _ = _run(g, order, v, transpose, kps.F32)
    assert normwise_error(got, want) <= 1e-5


@pytest.mark.parametrize("dt", [kps.F64, kps.F32])
def test_tie_group_longer_than_a_tile(dt):
    """45 hands that all tie (longer than one 32-hand tile): general kernel."""
    spec = synth.micro_spec(seed=19, ranks=5, suits=2, nboard=0)
    spec["strength"] = [1] * 45
    og, g = OracleGame(spec), kps.Game(spec)
    assert g.info()["max_tie"] == 45
    order = library_order(spec["strength"])
    for transpose in (False, True):
        v = _inputs(og, 3, seed=59, transpose=transpose)
        got, _ = _run(g, order, v, transpose, dt)
        want = og.matvec_AT(v) if transpose else og.matvec_A(v)
        assert normwise_error(got, want) <= TOL[dt]


@pytest.mark.parametrize("dt", [kps.F64, kps.F32])
def test_scalar_staging_path(river, dt, monkeypatch):
    """The non-vectorised fast path (used for half precision and for vectors
    that are not 16-byte aligned) on the river game."""
    spec, og, g, order = river
    monkeypatch.setenv("KPS_NO_VEC", "1")
    for transpose in (False, True):
        v = _inputs(og, 4, seed=61, transpose=transpose)
        got, _ = _run(g, order, v, transpose, dt)
        want = og.matvec_AT(v) if transpose else og.matvec_A(v)
        assert normwise_error(got, want) <= TOL[dt]


def test_unaligned_vectors(river):
    """Vectors starting 4 bytes into an allocation take the scalar staging path."""
    spec, og, g, order = river
    inf = g.info()
    B = 3
    y = _inputs(og, B, seed=67, transpose=False)
    yl = torch.from_numpy(to_library(y, order, inf["hs"])).to("cuda", torch.float32).reshape(-1)
    ybuf = torch.zeros(yl.numel() + 1, device="cuda")
    ybuf[1:] = yl
    obuf = torch.zeros(B * inf["n1"] * inf["hs"] + 1, device="cuda")
    kps.matvec_A(g, ybuf[1:], obuf[1:], B)
    torch.cuda.synchronize()
    o = obuf[1:].reshape(B, inf["n1"], inf["hs"]).double().cpu().numpy()
    assert normwise_error(from_library(o, order, inf["H"]), og.matvec_A(y)) <= 1e-5


@pytest.mark.parametrize("transpose", [False, True])
def test_flop_size_game_uses_spill_rows(transpose):
    """A 1176-hand game (3-card board): its four chunks of ~294 hands need the
    tiles cut from the chunk ends and the spill rows past the tensor-memory
    region; FP32 products within the FP32 bound of the oracle."""
    spec = synth.river_spec(seed=9, nboard=3)
    og, g = OracleGame(spec), kps.Game(spec)
    inf = g.info()
    assert inf["H"] == 1176
    order = library_order(spec["strength"])
    v = _inputs(og, 3, seed=67, transpose=transpose)
    n_out = inf["n2"] if transpose else inf["n1"]
    vin = torch.from_numpy(to_library(v, order, inf["hs"])).to("cuda", torch.float32).contiguous()
    out = torch.full((3, n_out, inf["hs"]), float("nan"), device="cuda")
    (kps.matvec_AT if transpose else kps.matvec_A)(g, vin, out, 3)
    torch.cuda.synchronize()
    got = from_library(out.double().cpu().numpy(), order, inf["H"])
    want = og.matvec_AT(v) if transpose else og.matvec_A(v)
    assert normwise_error(got, want) <= 1e-5
