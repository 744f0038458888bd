"""Host model of the output-sensitive pair listing (its rules restated with numpy FP32
arithmetic and explicit directed rounding), checked on random searches: no pair is listed
twice, and every pair that passes the FP32 filter of both of its rows (every pair within the
threshold does: the threshold's band covers the rounding of either form) is listed, in the row
whose site comes first in the bucket order. This pins the argument the CUDA kernel relies on;
the kernel itself is compared with the dense scan and the oracle in the GPU tests."""
import numpy as np
import pytest

f32 = np.float32
NB = 128


def rd(x64):   # round a float64 value down to float32
    r = f32(x64)
    return np.nextafter(r, f32(-np.inf)) if float(r) > x64 else r


def ru(x64):
    r = f32(x64)
    return np.nextafter(r, f32(np.inf)) if float(r) < x64 else r


def bucket(x, lo, inv):
    with np.errstate(invalid="ignore"):   # inf * 0 = NaN: the last bucket, as in the kernel
        f = f32(f32(x - lo) * inv)        # round to nearest, as the kernel
    return max(0, int(f)) if f < f32(NB) else NB - 1


def passes(a, s, J4, c, i, j):
    """Row i's FP32 test of pair {i, j}: fl(a_j + s_i s_j 4J~_ij) <= c_i."""
    return f32(a[j] + f32(s[i] * s[j]) * J4[i, j]) <= c[i]


def listing(a, s, J4, thr):
    n = a.size
    rm = np.abs(J4).max(axis=1).astype(f32)
    amin = a.min()
    c = (thr - a).astype(f32)
    live = [i for i in range(n) if c[i] >= rd(float(amin) - float(rm[i]))]
    if not live:
        return [], c
    t = {i: ru(float(np.nextafter(c[i], f32(np.inf))) + float(rm[i])) for i in live}
    B = max(t.values())
    span = ru(float(B) - float(amin))
    inv = f32(f32(NB) / span) if (span > 0 and np.isfinite(span)) else f32(0)
    cols = [j for j in range(n) if a[j] < B]
    order = sorted(cols, key=lambda j: bucket(a[j], amin, inv))   # any order within a bucket
    pos = {j: k for k, j in enumerate(order)}
    ends = np.cumsum(np.bincount([bucket(a[j], amin, inv) for j in cols], minlength=NB))
    pairs = []
    for i in live:
        if i not in pos:
            continue
        end = int(ends[bucket(t[i], amin, inv)])
        pairs += [(i, order[k]) for k in range(pos[i] + 1, end)]
    return pairs, c


@pytest.mark.parametrize("seed", range(6))
def test_listing_covers_every_pair_passing_both_rows(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(40, 160))
    J = np.triu(rng.standard_normal((n, n)), 1)
    J4 = (4 * (J + J.T)).astype(f32)
    s = rng.choice([-1.0, 1.0], n).astype(f32)
    a = (rng.standard_normal(n) * 8 + rng.uniform(-5, 5)).astype(f32)
    # a threshold that keeps a few percent of the pairs
    vals = np.array([float(a[i]) + float(a[j]) + float(s[i] * s[j] * J4[i, j]) for i in range(n) for j in range(i + 1, n)])
    thr = f32(np.quantile(vals, rng.uniform(0.005, 0.05)))
    pairs, c = listing(a, s, J4, thr)
    keys = [tuple(sorted(p)) for p in pairs]
    assert len(keys) == len(set(keys))   # each pair listed at most once
    listed = set(keys)
    both = [(i, j) for i in range(n) for j in range(i + 1, n)
            if passes(a, s, J4, c, i, j) and passes(a, s, J4, c, j, i)]
    assert both, "threshold keeps no pair"
    for p in both:
        assert p in listed
    # the listing is much smaller than all pairs at these thresholds
    assert len(pairs) < n * (n - 1) // 2


def test_infinite_threshold_lists_every_pair_once():
    rng = np.random.default_rng(9)
    n = 30
    J = np.triu(rng.standard_normal((n, n)), 1)
    J4 = (4 * (J + J.T)).astype(f32)
    s = rng.choice([-1.0, 1.0], n).astype(f32)
    a = rng.standard_normal(n).astype(f32)
    pairs, _ = listing(a, s, J4, f32(np.inf))
    assert sorted(tuple(sorted(p)) for p in pairs) == [(i, j) for i in range(n) for j in range(i + 1, n)]
