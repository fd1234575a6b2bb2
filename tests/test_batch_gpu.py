"""Batched products (one persistent launch over uneven games) against the
FP64 oracle, game by game.

The batch mixes river-shaped games with 3-, 4- and 5-card boards (1176,
1128, 1081 hands) and different betting trees with small games of a few
hands, so tiles of very different games meet in one launch.  Tolerances are
those of the single-game products (normwise 1e-12 FP64, 1e-5 FP32, 2^-8
BF16, 2^-10 FP16, half precision against the oracle on the same rounded
inputs).
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


def _specs():
    specs = synth.batch_specs(seed=11, n=4)
    specs.insert(1, synth.micro_spec(seed=5, ranks=4, suits=2, nboard=2))
    specs.append(synth.micro_spec(seed=6, ranks=5, suits=2, nboard=1, raise_cap=-1, stack=30.0))
    specs.insert(3, synth.micro_spec(seed=7, ranks=3, suits=2, nboard=0))
    return specs


@pytest.fixture(scope="module")
def batch():
    specs = _specs()
    games = [kps.Game(s) for s in specs]
    oracles = [OracleGame(s) for s in specs]
    orders = [library_order(s["strength"]) for s in specs]
    b = kps.Batch(games)
    # one random vector per game and player, and the oracle's products
    vec = {}
    for p in (0, 1):
        vs = []
        for i, og in enumerate(oracles):
            vs.append(synth.simplex_vectors(og.sequences(p)["nact"], og.H, 1, seed=100 * i + p)[0])
        vec[p] = vs
    want_A = [og.matvec_A(vec[1][i][None])[0] for i, og in enumerate(oracles)]
    want_AT = [og.matvec_AT(vec[0][i][None])[0] for i, og in enumerate(oracles)]
    return dict(specs=specs, games=games, oracles=oracles, orders=orders, b=b, vec=vec,
                want={0: want_A, 1: want_AT})


def _pack(bt, p, vecs, tdt):
    off = bt["b"].offsets(p)
    flat = np.zeros(off[-1])
    for i, g in enumerate(bt["games"]):
        hs = g.info()["hs"]
        v = to_library(vecs[i], bt["orders"][i], hs)
        flat[off[i]:off[i + 1]] = v.reshape(-1)
    return torch.from_numpy(flat).to("cuda", tdt)


def _unpack(bt, p, flat):
    off = bt["b"].offsets(p)
    out = []
    for i, g in enumerate(bt["games"]):
        inf = g.info()
        n = inf["n1"] if p == 0 else inf["n2"]
        v = flat[off[i]:off[i + 1]].reshape(n, inf["hs"])
        assert np.all(v[:, inf["H"]:] == 0), "padding must be written as zero"
        out.append(from_library(v, bt["orders"][i], inf["H"]))
    return out


def _check(bt, dt, transpose):
    p_in, p_out = (0, 1) if transpose else (1, 0)
    vin_canon = bt["vec"][p_in]
    vin = _pack(bt, p_in, vin_canon, TDT[dt])
    n_out = int(bt["b"].offsets(p_out)[-1])
    out = torch.full((n_out,), float("nan"), device="cuda", dtype=TDT[dt])
    (bt["b"].matvec_AT if transpose else bt["b"].matvec_A)(vin, out, dtype=dt)
    torch.cuda.synchronize()
    got = _unpack(bt, p_out, out.to(torch.float64).cpu().numpy())
    rounded = vin.to(torch.float64).cpu().numpy()
    for i, og in enumerate(bt["oracles"]):
        if dt in (kps.BF16, kps.F16):
            # the oracle on the same rounded inputs
            off = bt["b"].offsets(p_in)
            inf = bt["games"][i].info()
            n_in = inf["n2"] if p_in == 1 else inf["n1"]
            v = from_library(rounded[off[i]:off[i + 1]].reshape(n_in, inf["hs"]), bt["orders"][i], inf["H"])
            want = (og.matvec_AT if transpose else og.matvec_A)(v[None])[0]
        else:
            want = bt["want"][1 if transpose else 0][i]
        assert normwise_error(got[i], want) <= TOL[dt], f"game {i}"


@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("dt", [kps.F32, kps.BF16, kps.F16, kps.F64])
def test_batch_matches_oracle(batch, dt, transpose):
    _check(batch, dt, transpose)


@pytest.mark.parametrize("schedule", [0, 1])
def test_every_warp_count_and_schedule(batch, schedule):
    b = batch["b"]
    dflt = b.shape(kps.F32)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tried = 0
    for w in range(1, 9):
        try:
            b.set_shape(kps.F32, w, 3 if schedule else sms, schedule, kps.BATCH_TMEM)
        except kps.KpsError as e:
            assert e.status == kps.ENOTSUP
            continue
        tried += 1
        _check(batch, kps.F32, False)
        _check(batch, kps.F32, True)
    assert tried >= 2
    # the staged kernel runs 4 warps only, and not FP64
    for w in (3, 5):
        with pytest.raises(kps.KpsError) as e:
            b.set_shape(kps.F32, w, sms, schedule, kps.BATCH_STAGED)
        assert e.value.status == kps.ENOTSUP
    with pytest.raises(kps.KpsError) as e:
        b.set_shape(kps.F64, 4, sms, schedule, kps.BATCH_STAGED)
    assert e.value.status == kps.ENOTSUP
    with pytest.raises(kps.KpsError) as e:                  # at most two CTAs per SM
        b.set_shape(kps.F32, 4, 3 * sms, schedule, kps.BATCH_STAGED)
    assert e.value.status == kps.ENOTSUP
    try:
        b.set_shape(kps.F32, 4, 3 if schedule else 2 * sms, schedule, kps.BATCH_STAGED)
    except kps.KpsError as e:
        assert e.status == kps.ENOTSUP      # a game with a tie group over 4 hands
    else:
        assert b.shape(kps.F32)["kernel"] == kps.BATCH_STAGED
        _check(batch, kps.F32, False)
        _check(batch, kps.F32, True)
    b.set_shape(kps.F32, dflt["warps"], dflt["grid"], dflt["schedule"], dflt["kernel"])


def test_autotuner_picks_a_valid_shape(batch):
    b = batch["b"]
    for dt in (kps.F32, kps.F64):
        sh = b.tune(dt)
        assert 1 <= sh["warps"] <= 8 and sh["grid"] >= 1 and sh["schedule"] in (0, 1)
        assert sh["ms_per_pair"] > 0
        assert b.shape(dt)["warps"] == sh["warps"]
        _check(batch, dt, False)
        _check(batch, dt, True)


def test_batch_of_one_equals_single_game(batch):
    """A batch of one game runs the same arithmetic as kps_matvec_A with the
    same warp count: compare with the single-game product."""
    g = batch["games"][0]
    b1 = kps.Batch([g])
    inf = g.info()
    y = _pack(dict(batch, b=b1, games=[g], orders=batch["orders"][:1]), 1, batch["vec"][1][:1], torch.float32)
    out_b = torch.zeros(inf["n1"] * inf["hs"], device="cuda")
    b1.matvec_A(y, out_b)
    out_s = torch.zeros(1, inf["n1"], inf["hs"], device="cuda")
    kps.matvec_A(g, y.view(1, inf["n2"], inf["hs"]), out_s, 1)
    torch.cuda.synchronize()
    assert normwise_error(out_b.cpu().numpy(), out_s.view(-1).cpu().numpy()) <= 1e-6


def test_misaligned_and_mixed_batches_rejected(batch):
    g2 = batch["games"][0]
    one = kps.Game(synth.tiny_spec())   # one-card hands
    with pytest.raises(kps.KpsError) as e:
        kps.Batch([g2, one])
    assert e.value.status == kps.EINVAL
    b = batch["b"]
    n1, n2 = int(b.offsets(0)[-1]), int(b.offsets(1)[-1])
    y = torch.zeros(n2 + 4, device="cuda")
    out = torch.zeros(n1, device="cuda")
    with pytest.raises(kps.KpsError) as e:
        b.matvec_A(y[1:], out)     # 4-byte offset: not 16-byte aligned
    assert e.value.status == kps.EINVAL


def test_staged_kernel_leaves_long_ties_to_tensor_memory_kernel():
    """A game with a tie group of 5 hands is not taken by the staged kernel:
    the batch's default FP32 / BF16 / FP16 products run the staged kernel for
    the other games and the tensor-memory kernel for that one, and every game
    matches the oracle (half precision: on the rounded inputs)."""
    tied = synth.river_spec(seed=2)
    s = np.asarray(tied["strength"])
    order = np.lexsort((np.arange(len(s)), s))
    s = s.copy()
    s[order[100:105]] = s[order[100]]
    tied["strength"] = s.tolist()
    specs = [synth.river_spec(seed=3), tied, synth.river_spec(seed=4, nboard=4)]
    bt = {"specs": specs, "games": [kps.Game(x) for x in specs]}
    bt["oracles"] = [OracleGame(x) for x in specs]
    bt["orders"] = [library_order(x["strength"]) for x in specs]
    bt["b"] = kps.Batch(bt["games"])
    assert bt["b"].shape(kps.F32)["kernel"] == kps.BATCH_STAGED
    bt["vec"] = {p: [synth.simplex_vectors(og.sequences(p)["nact"], og.H, 1, seed=40 * i + p)[0]
                     for i, og in enumerate(bt["oracles"])] for p in (0, 1)}
    bt["want"] = {0: [og.matvec_A(bt["vec"][1][i][None])[0] for i, og in enumerate(bt["oracles"])],
                  1: [og.matvec_AT(bt["vec"][0][i][None])[0] for i, og in enumerate(bt["oracles"])]}
    for dt in (kps.F32, kps.BF16, kps.F16):
        assert bt["b"].shape(dt)["kernel"] == kps.BATCH_STAGED
        _check(bt, dt, False)
        _check(bt, dt, True)
