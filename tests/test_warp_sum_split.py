"""The split the kernels use for exact 64-bit warp sums (three 32-bit warp
reductions), emulated on the host: v = a 2^42 + b 2^21 + c with b, c in
[0, 2^21) and a in [-2^21, 2^21); the three part sums of 32 lanes fit 32 bits
and recombine to the 64-bit sum modulo 2^64, for any lane values, including
the extremes and mixed signs."""
import numpy as np

MASK = (1 << 21) - 1


def _split_sum(vals):
    v = [int(x) for x in vals]
    c = [x & MASK for x in v]
    b = [(x >> 21) & MASK for x in v]
    a = [x >> 42 for x in v]  # arithmetic shift of a signed 64-bit value
    assert all(-(1 << 21) <= x < (1 << 21) for x in a)
    sc, sb = sum(c) % (1 << 32), sum(b) % (1 << 32)
    sa = sum(a) % (1 << 32)
    sa = sa - (1 << 32) if sa >= (1 << 31) else sa  # the 32-bit sum read as signed
    assert sum(c) < (1 << 32) and sum(b) < (1 << 32) and abs(sum(a)) < (1 << 31)
    t = (sa * (1 << 42) + sb * (1 << 21) + sc) % (1 << 64)
    return t - (1 << 64) if t >= (1 << 63) else t


def _ref(vals):
    t = sum(int(x) for x in vals) % (1 << 64)
    return t - (1 << 64) if t >= (1 << 63) else t


def test_split_sum_is_exact():
    rng = np.random.default_rng(0)
    cases = [rng.integers(-(1 << 63), (1 << 63) - 1, 32, dtype=np.int64, endpoint=True) for _ in range(200)]
    cases += [rng.integers(-(1 << 40), 1 << 40, 32, dtype=np.int64) for _ in range(200)]
    cases += [np.full(32, -(1 << 63), np.int64), np.full(32, (1 << 63) - 1, np.int64), np.zeros(32, np.int64),
              np.array([-1] * 31 + [1], np.int64), np.array([(1 << 42) - 1, -(1 << 42)] * 16, np.int64)]
    for v in cases:
        assert _split_sum(v) == _ref(v)
