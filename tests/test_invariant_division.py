"""Pin of the division by an invariant integer used by the two-stage
partner choice (Granlund and Montgomery 1994, Fig. 4.1): for 2 <= d < 2^17,
l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1 and t = floor(m x / 2^32),
the quotient floor(x / d) equals (t + floor((x - t) / 2)) >> (l - 1) for
every 32-bit x.  Checked exhaustively over d at the x that stress it (0, 1,
multiples of d and their neighbours, 2^32 - 1) and on random x."""
import numpy as np


def _magic(d):
    l = 0
    while (1 << l) < d:
        l += 1
    return ((1 << 32) * ((1 << l) - d)) // d + 1, l - 1


def _div(x, m, s):
    t = (m * x) >> 32
    return (t + ((x - t) >> 1)) >> s


def test_invariant_division_is_exact():
    rng = np.random.default_rng(5)
    ds = list(range(2, 4097)) + [int(d) for d in rng.integers(4097, 65538, 3000)] + [32768, 32769, 65536, 65537]
    for d in ds:
        m, s = _magic(d)
        assert 0 < m < (1 << 32)
        xs = [0, 1, d - 1, d, d + 1, (1 << 32) - 1, (1 << 32) - d, ((1 << 32) - 1) // d * d,
              ((1 << 32) - 1) // d * d - 1] + [int(x) for x in rng.integers(0, 1 << 32, 8, dtype=np.uint64)]
        for x in xs:
            assert _div(x, m, s) == x // d, (d, x)
