"""Helpers shared by the GPU parity tests: layout conversion between the
oracle's canonical [seq][hand] vectors and the library's strength-ordered,
padded [seq][hs] vectors, and the normwise error used throughout."""
import numpy as np


def library_order(strength):
    """Ascending strength, ties by canonical index (the ABI's hand order)."""
    s = np.asarray(strength)
    return np.lexsort((np.arange(len(s)), s))


def to_library(v, order, hs):
    """[B][n][H] canonical -> [B][n][hs] library order, zero padded."""
    v = np.asarray(v)
    out = np.zeros(v.shape[:-1] + (hs,), dtype=v.dtype)
    out[..., :v.shape[-1]] = v[..., order]
    return out


def from_library(v, order, H):
    """[B][n][hs] library order -> [B][n][H] canonical."""
    v = np.asarray(v)
    out = np.zeros(v.shape[:-1] + (H,), dtype=v.dtype)
    out[..., order] = v[..., :H]
    return out


def normwise_error(got, want):
    """max |got - want| / max |want| (the error measure for products whose
    entries cancel: win and lose mass subtract)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = np.max(np.abs(want))
    if scale == 0:
        return float(np.max(np.abs(got)))
    return float(np.max(np.abs(got - want)) / scale)
