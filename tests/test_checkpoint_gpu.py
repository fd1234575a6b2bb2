"""Checkpoint / resume and non-finite detection at the C ABI.

* A solver checkpointed after k iterations and loaded into a fresh solver
  (which had run other iterations first) continues bit for bit like the
  solver that never stopped: the whole saved state after the same further
  iterations is identical byte for byte, for RM+ and Discounted CFR, in
  FP64, FP32 and BF16 storage.
* Loading a checkpoint into a solver of another batch or storage type, or
  from a truncated buffer, is refused with KPS_EINVAL.
* A NaN in a caller-prepared initial strategy is caught by the check that
  follows every kps_solver_step: KPS_ENUMERIC from kps_solver_status and
  from later steps, until the solver is reset.
* The warm-start network checkpointed after some Adam steps and loaded into
  a network with another initialisation takes the same further steps, bit
  for bit (parameters, moments and step count are all restored).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2112_03804_gb300 import kps, synth

pytestmark = pytest.mark.gpu


def _batch():
    specs = [synth.micro_spec(seed=3), synth.river_spec(seed=5), synth.micro_spec(seed=8, ranks=5),
             synth.river_spec(seed=6, nboard=4)]
    return kps.Batch([kps.Game(s) for s in specs])


@pytest.mark.parametrize("method", [0, 1], ids=["rmplus", "dcfr"])
@pytest.mark.parametrize("dt", [kps.F64, kps.F32, kps.BF16])
def test_solver_resume_is_bit_identical(dt, method):
    b = _batch()
    a = kps.Solver(b, dt)
    if method == 1:
        a.set_method(1, 1.5, 0.0, 2.0)
    a.reset()
    a.step(7)
    ck = a.save()
    a.step(5)
    want = a.save()
    a.status()

    fresh = kps.Solver(b, dt)
    fresh.step(3)                      # state the checkpoint must replace
    fresh.load(ck)
    assert fresh.iterations() == 7
    fresh.step(5)
    got = fresh.save()
    fresh.status()
    assert got == want

    n = len(b.games)
    ea = torch.zeros(n, dtype=torch.float64, device="cuda")
    eb = torch.zeros(n, dtype=torch.float64, device="cuda")
    a.exploitability(ea)
    fresh.exploitability(eb)
    torch.cuda.synchronize()
    assert torch.equal(ea, eb)


def test_load_rejects_mismatches():
    b = _batch()
    s = kps.Solver(b, kps.F32)
    s.step(2)
    ck = s.save()
    other = kps.Solver(kps.Batch([kps.Game(synth.micro_spec(seed=4))]), kps.F32)
    with pytest.raises(kps.KpsError) as e:
        other.load(ck)
    assert e.value.status == kps.EINVAL
    wide = kps.Solver(b, kps.F64)
    with pytest.raises(kps.KpsError) as e:
        wide.load(ck)
    assert e.value.status == kps.EINVAL
    with pytest.raises(kps.KpsError) as e:
        s.load(ck[: len(ck) // 2])
    assert e.value.status == kps.EINVAL
    with pytest.raises(kps.KpsError) as e:
        s.load(b"\0" * len(ck))
    assert e.value.status == kps.EINVAL
    s.load(ck)
    s.step(1)
    s.status()


def test_nan_in_initial_strategy_is_reported():
    b = kps.Batch([kps.Game(synth.micro_spec(seed=3)), kps.Game(synth.micro_spec(seed=5))])
    s = kps.Solver(b, kps.F32)
    x = torch.zeros(int(b.offsets(0)[-1]), dtype=torch.float64, device="cuda")
    y = torch.zeros(int(b.offsets(1)[-1]), dtype=torch.float64, device="cuda")
    s.average(x, y, behavioural=True)           # uniform behavioural strategies
    beh1, beh2 = x.float(), y.float()
    s.reset(beh1, beh2)
    s.step(3)
    s.status()                                   # a finite start passes
    bad = beh1.clone()
    bad[1] = float("nan")
    s.reset(bad, beh2)
    s.step(3)
    with pytest.raises(kps.KpsError) as e:
        s.status()
    assert e.value.status == kps.ENUMERIC
    with pytest.raises(kps.KpsError) as e:
        s.step(1)
    assert e.value.status == kps.ENUMERIC
    s.reset()
    s.step(3)
    s.status()


def _training_data(rows, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    X = torch.rand((rows, kps.WARM_DIN), device="cuda", generator=g)
    nact = torch.randint(2, kps.WARM_DOUT + 1, (rows,), device="cuda", generator=g, dtype=torch.int32)
    T = torch.rand((rows, kps.WARM_DOUT), device="cuda", generator=g)
    mask = torch.arange(kps.WARM_DOUT, device="cuda")[None, :] < nact[:, None]
    T = torch.where(mask, T, torch.zeros_like(T))
    T = T / T.sum(dim=1, keepdim=True)
    w = torch.rand(rows, device="cuda", generator=g) + 0.5
    return X, nact, T, w


def test_mlp_resume_is_bit_identical():
    rows = 300
    data = [_training_data(rows, seed) for seed in range(5)]
    m = kps.MLP(seed=0)

    def step(net, k):
        X, nact, T, w = data[k]
        net.gradients(X, rows, nact, T, w, float(w.sum()))
        net.adam(1e-3)

    for k in range(3):
        step(m, k)
    ck = m.save()
    for k in (3, 4):
        step(m, k)
    torch.cuda.synchronize()
    want = m.save()

    other = kps.MLP(seed=7)
    step(other, 0)
    other.load(ck)
    for k in (3, 4):
        step(other, k)
    torch.cuda.synchronize()
    assert other.save() == want
    assert np.array_equal(other.get(0), m.get(0))
    small = kps.MLP(width=128, seed=1)
    with pytest.raises(kps.KpsError) as e:
        small.load(ck)
    assert e.value.status == kps.EINVAL
