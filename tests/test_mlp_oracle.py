"""Pins of the network oracle (oracle/mlp_oracle.py), CPU only.

* The analytic gradient equals central finite differences of the loss (an
  independent evaluation: only the forward definition is shared), for every
  parameter block, on a small network with ReLUs active and inactive and
  rows with different action counts.
* With all weights zero the network is its output bias: P is the softmax of
  b3 over the node's actions (closed form [1,2,3]/6 and [1,2,3,4]/10 for
  b3 = log(1..4)), the loss is the cross-entropy of those, the gradient of
  b3 is sum_q w_q (P_q - T_q) / sum w, masked actions have P = 0 and zero
  gradient, and every weight gradient is zero (the hidden layers are 0).
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def _problem(seed=0, din=7, width=5, dout=4, Q=6):
    r = np.random.default_rng(seed)
    n = sum(int(np.prod(s)) for s in M.shapes(din, width, dout))
    params = r.normal(0, 0.7, size=n)
    X = r.normal(0, 1, size=(Q, din))
    nact = r.integers(2, dout + 1, size=Q)
    T = np.zeros((Q, dout))
    for q in range(Q):
        T[q, :nact[q]] = r.dirichlet(np.ones(nact[q]))
    w = r.uniform(0.2, 2.0, size=Q)
    return params, X, nact, T, w, (din, width, dout)


def test_gradient_matches_finite_differences():
    params, X, nact, T, w, dims = _problem()
    L, g = M.loss_and_grads(params, X, nact, T, w, *dims)
    h = 1e-6
    num = np.zeros_like(params)
    for i in range(len(params)):
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        num[i] = (M.loss(p1, X, nact, T, w, *dims) - M.loss(p2, X, nact, T, w, *dims)) / (2 * h)
    assert np.max(np.abs(num - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))
    # some ReLUs are inactive, so the check covers both branches
    _, (_, A1, _, A2, _, _) = M.forward(params, X, nact, *dims)
    assert (A1 < 0).any() and (A1 > 0).any() and (A2 < 0).any() and (A2 > 0).any()


def test_zero_weights_closed_forms():
    din, width, dout = 3, 4, 4
    blocks = [np.zeros(s) for s in M.shapes(din, width, dout)]
    blocks[5] = np.log(np.array([1.0, 2.0, 3.0, 4.0]))
    params = M.pack(blocks)
    X = np.ones((2, din))
    nact = np.array([3, 4])
    T = np.array([[1.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0, 1.0]])
    w = np.array([1.0, 3.0])
    P, _ = M.forward(params, X, nact, din, width, dout)
    assert np.allclose(P[0], [1 / 6, 2 / 6, 3 / 6, 0.0], rtol=0, atol=1e-15)
    assert np.allclose(P[1], [0.1, 0.2, 0.3, 0.4], rtol=0, atol=1e-15)
    L, g = M.loss_and_grads(params, X, nact, T, w, din, width, dout)
    assert L == pytest.approx(-(1.0 * np.log(1 / 6) + 3.0 * np.log(0.4)) / 4.0, rel=1e-14)
    gW1, gb1, gW2, gb2, gW3, gb3 = M.unpack(g, din, width, dout)
    expect = (1.0 * (np.array([1 / 6, 2 / 6, 3 / 6, 0.0]) - T[0])
              + 3.0 * (np.array([0.1, 0.2, 0.3, 0.4]) - T[1])) / 4.0
    expect_masked = expect.copy()
    # row 0 has 3 actions: its 4th output contributes nothing
    expect_masked[3] = 3.0 * (0.4 - 1.0) / 4.0
    assert np.allclose(gb3, expect_masked, atol=1e-15)
    for blk in (gW1, gb1, gW2, gb2, gW3):
        assert np.all(blk == 0.0)
