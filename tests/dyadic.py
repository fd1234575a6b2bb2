"""Games whose products are exact in FP32: beliefs that make beta a power of
four (lambda = mu / sqrt(beta) dyadic), so that with small-integer vectors and
dyadic payoffs every sum the kernels form is exact and the GPU must equal
the FP64 oracle bit for bit.  Host-side helpers for the GPU tests (random
draws and a search over belief choices; none of the method's arithmetic).
"""
import numpy as np

from paper_2112_03804_gb300 import synth


def hand_cards(spec):
    """Card pairs of the canonical hand order (deck minus board, a < b)."""
    left = [c for c in range(spec["ranks"] * spec["suits"]) if c not in set(spec["board"])]
    return [(a, b) for i, a in enumerate(left) for b in left[i + 1:]]


def dyadic_beliefs(spec, seed):
    """mu1 in {1, 2}, mu2 in {0, 1} with beta = sum over compatible pairs of
    mu1 mu2 = 2^20, so lambda = mu / 2^10 is exact in FP32."""
    cards = np.array(hand_cards(spec))
    H = len(cards)
    ind = np.zeros((H, spec["ranks"] * spec["suits"]), dtype=np.int64)
    ind[np.arange(H), cards[:, 0]] = 1
    ind[np.arange(H), cards[:, 1]] = 1
    compat = (ind @ ind.T) == 0
    r = np.random.default_rng(seed)
    mu1 = np.ones(H)
    mu1[r.choice(H, 300, replace=False)] = 2.0
    c1 = (compat * mu1[:, None]).sum(axis=0).astype(np.int64)   # per player-2 hand
    rem = int(c1.sum()) - (1 << 20)
    k = int(round(rem / c1.mean()))
    out = list(r.choice(H, k, replace=False))
    inside = np.zeros(H, dtype=bool)
    inside[out] = True
    for _ in range(10000):
        diff = rem - int(c1[inside].sum())
        if diff == 0:
            break
        # one swap that moves the removed sum towards the target
        a = np.flatnonzero(inside)
        b = np.flatnonzero(~inside)
        gain = c1[b][None, :] - c1[a][:, None]
        i, j = np.unravel_index(np.argmin(np.abs(gain - diff)), gain.shape)
        if abs(int(gain[i, j]) - diff) >= abs(diff):
            raise AssertionError("no improving swap")
        inside[a[i]] = False
        inside[b[j]] = True
    assert int(c1[inside].sum()) == rem
    mu2 = np.where(inside, 0.0, 1.0)
    beta = float((compat * np.outer(mu1, mu2)).sum())
    assert beta == float(1 << 20)
    return mu1.tolist(), mu2.tolist()


def grouped_strengths(spec, seed):
    """Strength order of the spec, then consecutive hands merged into tie
    groups of 1 to 4 hands."""
    s = np.asarray(spec["strength"])
    order = np.lexsort((np.arange(len(s)), s))
    r = np.random.default_rng(seed)
    out = np.empty(len(s), dtype=np.int64)
    pos, gid = 0, 0
    while pos < len(s):
        n = int(r.integers(1, 5))
        out[order[pos:pos + n]] = gid
        pos += n
        gid += 1
    return out.tolist()


def dyadic_river(seed, ties, nboard=5):
    """A river-shaped game (nboard-card board) with dyadic lambda; with
    ties, every hand in a tie group of 1 to 4 hands."""
    spec = synth.river_spec(seed=seed, nboard=nboard)
    if ties:
        spec["strength"] = grouped_strengths(spec, seed + 100)
    spec["mu1"], spec["mu2"] = dyadic_beliefs(spec, seed + 200)
    return spec
