"""Oracle of the warm-start network: plain FP64 numpy, test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline use this
module; the library never calls it.  The network is the definition written
out, layer by layer, with no fusion:

    H1 = relu(X W1 + b1),  H2 = relu(H1 W2 + b2),  Z = H2 W3 + b3
    P[q, a] = exp(Z[q, a]) / sum_{a' < nact[q]} exp(Z[q, a'])   (a < nact[q]), 0 otherwise
    L = - sum_q w[q] sum_{a < nact[q]} T[q, a] log P[q, a] / sum_q w[q]

and its gradient by the chain rule.  The flat parameter order is W1
[din][width], b1, W2 [width][width], b2, W3 [width][dout], b3.  Pinned by
central finite differences of L and by closed forms with zero weights
(tests/test_mlp_oracle.py).  The warm start itself has no counterpart in the
paper.
"""
from __future__ import annotations

import numpy as np


def shapes(din: int, width: int, dout: int):
    return [(din, width), (width,), (width, width), (width,), (width, dout), (dout,)]


def unpack(params, din: int, width: int, dout: int):
    out, o = [], 0
    for sh in shapes(din, width, dout):
        n = int(np.prod(sh))
        out.append(np.asarray(params[o:o + n], dtype=np.float64).reshape(sh))
        o += n
    return out


def pack(blocks) -> np.ndarray:
    return np.concatenate([np.asarray(b, dtype=np.float64).reshape(-1) for b in blocks])


def _masked_softmax(Z, nact):
    P = np.zeros_like(Z)
    for q in range(Z.shape[0]):
        z = Z[q, :nact[q]]
        e = np.exp(z - z.max())
        P[q, :nact[q]] = e / e.sum()
    return P


def forward(params, X, nact, din, width, dout):
    W1, b1, W2, b2, W3, b3 = unpack(params, din, width, dout)
    X = np.asarray(X, dtype=np.float64)
    A1 = X @ W1 + b1
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ W2 + b2
    H2 = np.maximum(A2, 0.0)
    Z = H2 @ W3 + b3
    P = _masked_softmax(Z, nact)
    return P, (X, A1, H1, A2, H2, Z)


def loss(params, X, nact, T, w, din, width, dout) -> float:
    P, _ = forward(params, X, nact, din, width, dout)
    T = np.asarray(T, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    total = 0.0
    for q in range(P.shape[0]):
        na = nact[q]
        t, p = T[q, :na], P[q, :na]
        m = t > 0
        total -= w[q] * np.sum(t[m] * np.log(p[m]))
    return total / w.sum()


def loss_and_grads(params, X, nact, T, w, din, width, dout):
    W1, b1, W2, b2, W3, b3 = unpack(params, din, width, dout)
    P, (X, A1, H1, A2, H2, Z) = forward(params, X, nact, din, width, dout)
    T = np.asarray(T, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    ws = w.sum()
    # dL/dZ: w_q (P - T) / sum w on the node's actions, 0 elsewhere
    dZ = np.zeros_like(Z)
    for q in range(Z.shape[0]):
        na = nact[q]
        dZ[q, :na] = w[q] * (P[q, :na] - T[q, :na]) / ws
    gW3 = H2.T @ dZ
    gb3 = dZ.sum(axis=0)
    dH2 = dZ @ W3.T
    dA2 = dH2 * (A2 > 0)
    gW2 = H1.T @ dA2
    gb2 = dA2.sum(axis=0)
    dH1 = dA2 @ W2.T
    dA1 = dH1 * (A1 > 0)
    gW1 = X.T @ dA1
    gb1 = dA1.sum(axis=0)
    L = loss(params, X, nact, T, w, din, width, dout)
    return L, pack([gW1, gb1, gW2, gb2, gW3, gb3])
