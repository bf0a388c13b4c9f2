"""The exact six-way BF16 slicing behind the tensor-core contractions (the build's
G Q products and the W form), replayed in float32 on the CPU: a float pair scaled to
|h + l| < 32 is cut into integer slices d_0..d_5 (weights 2^-8u) by round, subtract and
multiply-by-256 steps, the low word from slice 3 on.  Checked: every slice is an
integer that BF16 holds exactly, within the stated bounds, the slices sum to the pair
within 2^-40 of the scale, and a 64-long sum of slice products on any diagonal stays
below 2^24, where FP32 accumulation of integers is exact.  The pose kernels' five-slice
form (weights stored with the slices, two accumulators) is replayed the same way."""
import numpy as np

F = np.float32


def slice6(h, l):
    d = []
    r = h.astype(F)
    for _ in range(6):
        q = np.rint(r).astype(F)
        d.append(q)
        r = ((r - q).astype(F) * F(256)).astype(F)
    r = (l.astype(F) * F(16777216.0)).astype(F)  # l in units of slice 3 (2^-24)
    for u in range(3, 6):
        q = np.rint(r).astype(F)
        d[u] = (d[u] + q).astype(F)
        r = ((r - q).astype(F) * F(256)).astype(F)
    return d


def _pairs(rng, m):
    x = rng.uniform(-32.0, 32.0, m) * 10.0 ** rng.uniform(-3, 0, m)
    x = np.clip(x, -31.999, 31.999)
    h = x.astype(F)
    l = (x - h.astype(np.float64)).astype(F)
    return h, l


def _bf16_exact(v):
    b = np.asarray(v, dtype=F).view(np.uint32)
    return np.all((b & 0xFFFF) == 0)


def test_slices_are_bounded_bf16_integers_and_sum_to_the_pair():
    rng = np.random.default_rng(0)
    h, l = _pairs(rng, 200000)
    d = slice6(h, l)
    bounds = [32, 128, 128, 144, 256, 256]
    for u in range(6):
        assert np.all(d[u] == np.rint(d[u]))
        assert np.abs(d[u]).max() <= bounds[u]
        assert _bf16_exact(d[u])
    s = sum(d[u].astype(np.float64) * 2.0 ** (-8 * u) for u in range(6))
    x = h.astype(np.float64) + l.astype(np.float64)
    assert np.abs(s - x).max() <= 32.0 * 2.0 ** -40


def test_diagonal_sums_stay_exact_in_fp32():
    # the largest product on a diagonal u + v <= 5, over a 64-long K chunk
    bounds = [32, 128, 128, 144, 256, 256]
    worst = max(64 * sum(bounds[u] * bounds[dd - u] for u in range(dd + 1)) for dd in range(6))
    assert worst < 2 ** 24
    # and summing such products in float32 in any order is exact
    rng = np.random.default_rng(1)
    h, l = _pairs(rng, 64 * 2000)
    g, m = _pairs(rng, 64 * 2000)
    a, b = slice6(h, l), slice6(g, m)
    for dd in range(6):
        prod = sum(a[u].astype(np.float64) * b[dd - u].astype(np.float64) for u in range(dd + 1))
        prod = prod.reshape(2000, 64)
        acc = np.zeros(2000, dtype=F)
        for k in range(64):
            acc = (acc + prod[:, k].astype(F)).astype(F)
        assert np.array_equal(acc.astype(np.float64), prod.sum(axis=1))


def slice5(h, l):
    """The pose kernels' five slices (weights included), the low word joining at slice 2
    through one fused multiply-add."""
    d0 = np.rint(h).astype(F)
    t = ((h - d0).astype(F) * F(256)).astype(F)
    d1 = np.rint(t).astype(F)
    # fma: (t - d1) * 256 + l * 2^16 with one rounding
    t = (((t - d1).astype(F).astype(np.float64) * 256.0) + (l.astype(F) * F(65536.0)).astype(np.float64)).astype(F)
    d2 = np.rint(t).astype(F)
    t = ((t - d2).astype(F) * F(256)).astype(F)
    d3 = np.rint(t).astype(F)
    t = ((t - d3).astype(F) * F(256)).astype(F)
    d4 = np.rint(t).astype(F)
    return [d0, d1, d2, d3, d4]


def test_pose_kernel_five_slices():
    rng = np.random.default_rng(2)
    h, l = _pairs(rng, 200000)
    d = slice5(h, l)
    for u, b in enumerate([32, 128, 128, 128, 128]):
        assert np.all(d[u] == np.rint(d[u]))
        assert np.abs(d[u]).max() <= b
        assert _bf16_exact(d[u] * F(2.0 ** (-8 * u)))  # stored with its weight
    s = sum(d[u].astype(np.float64) * 2.0 ** (-8 * u) for u in range(5))
    x = h.astype(np.float64) + l.astype(np.float64)
    assert np.abs(s - x).max() <= 32.0 * 2.0 ** -37
    # diagonals 0 and 1 over a K of 32 stay exact multiples of 2^-8 below 2^24 of them
    assert 32 * (32 * 32 + 2 * 32 * 128) < 2 ** 24
