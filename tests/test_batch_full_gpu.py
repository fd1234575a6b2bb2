"""The batched launch at the shapes the benchmark times, against the oracle.

* The exact 4096-game batch of `bench.py --workload batch` (boards of 3-5
  cards, 1176/1128/1081 hands, trees of 13-209 terminals, one FP32 vector
  per game and player), launched with the autotuner's shape: 96 sampled
  entries of A y and of A^T x, each computed one by one by the FP64 oracle
  of its game, within the FP32 bound (normwise against that game's largest
  output, 1e-5).  Flop-size games (1176 hands) need the spill rows, so the
  launch runs the spill instantiation.  Checked with the tuned shape and
  with each of the two batched kernels (the staged one's chunks of 18-19
  boxes put their last boxes in its scratch area).
* A batch of river-shaped games with dyadic lambda (beta = 2^20; tests/
  dyadic.py) and small-integer vectors, on every launch shape the batch
  accepts (both kernels, warps per CTA, one or two CTAs per SM, ticket or
  static schedule; kps_batch_shape_set refuses the others): every
  FP32 product is exact, so the batched kernels must equal the oracle bit
  for bit, chunks of 1081 to 1176 hands with their tensor-memory region and
  spill rows included.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import kps, synth
from tests.dyadic import dyadic_river
from tests.gpu_util import from_library, library_order, to_library

pytestmark = pytest.mark.gpu


def _vectors(games, b, p, make):
    off = b.offsets(p)
    flat = np.zeros(int(off[-1]), dtype=np.float64)
    per = []
    for i, g in enumerate(games):
        inf = g.info()
        v = make(i, g, inf)                      # [n][H], library hand order
        per.append(v)
        w = np.zeros((v.shape[0], inf["hs"]))
        w[:, :inf["H"]] = v
        flat[off[i]:off[i + 1]] = w.reshape(-1)
    return flat, per


def test_full_benchmark_batch_sampled_entries():
    specs = synth.batch_specs(seed=4, n=4096)
    games = [kps.Game(s) for s in specs]
    b = kps.Batch(games)
    assert any(g.info()["H"] == 1176 for g in games)
    vec, per = {}, {}
    for p in (0, 1):
        flat, per[p] = _vectors(games, b, p, lambda i, g, inf: synth.simplex_vectors(
            g.sequences(p)["nact"], inf["H"], 1, seed=11 * i + p, dtype=np.float32)[0].astype(np.float64))
        vec[p] = torch.from_numpy(flat.astype(np.float32)).cuda()
    shape = b.tune(kps.F32)
    assert shape["warps"] >= 1
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # the tuned shape, then each kernel with two CTAs per SM
    for kernel in (None, kps.BATCH_STAGED, kps.BATCH_TMEM):
        if kernel is not None:
            b.set_shape(kps.F32, 4, 2 * sms, 0, kernel)
            assert b.shape(kps.F32)["kernel"] == kernel
        _sampled_entries(specs, games, b, vec, per, seed=23 + (kernel or 0))


def _sampled_entries(specs, games, b, vec, per, seed):
    out = {p: torch.full((int(b.offsets(p)[-1]),), float("nan"), device="cuda") for p in (0, 1)}
    b.matvec_A(vec[1], out[0])
    b.matvec_AT(vec[0], out[1])
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    for direction in (0, 1):                     # 0: A y (player-1 rows), 1: A^T x
        res = out[direction].double().cpu().numpy()
        off = b.offsets(direction)
        picks = rng.choice(len(games), size=96, replace=False)
        for i in picks:
            spec, g = specs[i], games[i]
            inf = g.info()
            n_out = inf["n1"] if direction == 0 else inf["n2"]
            got_game = res[off[i]:off[i + 1]].reshape(n_out, inf["hs"])
            assert np.all(got_game[:, inf["H"]:] == 0)
            og = OracleGame(spec)
            order = library_order(spec["strength"])
            s = int(rng.integers(n_out))
            hcan = int(rng.integers(inf["H"]))
            hlib = int(np.argsort(order)[hcan])
            vin = per[1 - direction][i]                       # library order
            vcan = np.zeros_like(vin)
            vcan[:, order] = vin
            want = og.matvec_entries(vcan[None], [0], [s], [hcan], transpose=direction == 1)[0]
            scale = float(np.max(np.abs(got_game[:, :inf["H"]])))
            assert abs(got_game[s, hlib] - want) <= 1e-5 * scale, (i, direction, s, hcan)


def test_dyadic_batch_bit_exact_every_shape():
    specs = [dyadic_river(seed=40 + k, ties=k % 2 == 1, nboard=nb) for k, nb in enumerate((5, 4, 3, 5, 3, 4))]
    games = [kps.Game(s) for s in specs]
    oracles = [OracleGame(s) for s in specs]
    orders = [library_order(s["strength"]) for s in specs]
    b = kps.Batch(games)
    vec, per = {}, {}
    for p in (0, 1):
        flat, per[p] = _vectors(games, b, p, lambda i, g, inf: synth.integer_vectors(
            inf["n1"] if p == 0 else inf["n2"], inf["H"], 1, seed=70 + 2 * i + p)[0])
        vec[p] = torch.from_numpy(flat.astype(np.float32)).cuda()
    want = {}
    for direction in (0, 1):
        want[direction] = []
        for i, og in enumerate(oracles):
            vcan = np.zeros_like(per[1 - direction][i])
            vcan[:, orders[i]] = per[1 - direction][i]
            want[direction].append((og.matvec_AT(vcan[None]) if direction == 1 else og.matvec_A(vcan[None]))[0])
    ran = 0
    shapes = [(kps.BATCH_TMEM, w) for w in range(1, 9)] + [(kps.BATCH_STAGED, 4)]
    for kernel, warps in shapes:
        for per_sm in (1, 2):
            for sched in (0, 1):
                try:
                    b.set_shape(kps.F32, warps=warps, grid=152 * per_sm, schedule=sched, kernel=kernel)
                except kps.KpsError as e:
                    assert e.status == kps.ENOTSUP and kernel == kps.BATCH_TMEM
                    continue
                out = {p: torch.full((int(b.offsets(p)[-1]),), float("nan"), device="cuda") for p in (0, 1)}
                b.matvec_A(vec[1], out[0])
                b.matvec_AT(vec[0], out[1])
                torch.cuda.synchronize()
                for direction in (0, 1):
                    res = out[direction].double().cpu().numpy()
                    off = b.offsets(direction)
                    for i in range(len(games)):
                        inf = games[i].info()
                        n_out = inf["n1"] if direction == 0 else inf["n2"]
                        got = from_library(res[off[i]:off[i + 1]].reshape(n_out, inf["hs"]), orders[i], inf["H"])
                        assert np.array_equal(got, want[direction][i]), (warps, per_sm, sched, direction, i)
                ran += 1
    assert ran >= 8
