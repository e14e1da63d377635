"""The fixed-point scale of the deterministic environment-gradient sums.

Per call the scale is 2^k with k = 62 - c - e, where 2^(e-1) <= 32 (V + 1) m
< 2^e (m: the largest |dL/d rgb| of a record, in float32; V: the most views
of a scene; 2^c >= 8 (surfels + records) + 1 contributions a texel can
receive).  A contribution is at most (V + 1) m; contributions above
2^(62 - c) after scaling are flagged rather than summed.  Checked here on the
CPU for the rule as the kernels state it: no sum of 2^c contributions leaves
63 bits, a contribution up to 16 times the bound is still summed, and one
unit is at most 2^(c - 56) (V + 1) m (about 2^-24 m for 1M surfels x 16
views)."""
import math

import numpy as np


def exponent(m, vmax, cbits):
    """k of the scale 2^k (0 for no contribution or a non-finite record)."""
    m = np.float32(m)
    if not (m > 0) or not (m < np.float32(1e30)):
        return 0
    _, e = math.frexp(float(np.float32(m * np.float32(32 * (vmax + 1)))))
    return 62 - cbits - e


def test_no_sum_leaves_63_bits_and_the_unit_is_bounded():
    rng = np.random.default_rng(91)
    for _ in range(20000):
        m = float(np.float32(math.exp(rng.uniform(math.log(1e-30), math.log(1e29)))))
        vmax = int(rng.integers(1, 257))
        cbits = int(rng.integers(1, 41))
        k = exponent(m, vmax, cbits)
        lim = 2.0 ** (62 - cbits)                       # a larger scaled contribution is flagged
        bound = (vmax + 1) * m * 2.0 ** k               # the largest contribution, scaled
        assert 16 * bound < lim                         # 16x headroom below the flag
        assert 2 ** cbits * lim <= 2.0 ** 62            # 2^c contributions below the limit fit int64
        assert 2.0 ** -k <= 2.0 ** (cbits - 56) * (vmax + 1) * m * (1 + 1e-6)


def test_headline_batch_unit():
    """1M surfels, 16 views: c = ceil(log2(8 * 17M + 1)) = 28, V = 16."""
    cbits = math.ceil(math.log2(8 * (1_000_000 + 16_000_000) + 1))
    assert cbits == 28
    for m in (1e-6, 0.37, 3.0, 1234.5):
        unit = 2.0 ** -exponent(m, 16, cbits) / float(np.float32(m))
        assert 2.0 ** -25 < unit <= 2.0 ** -23.9
