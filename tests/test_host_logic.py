"""Host-side logic that needs no GPU: the flat-index codec formula the
library uses, against the oracle's independent integer bisection."""
import numpy as np


def pair_from_index(qs):
    # the library's FP64 square root plus integer fix-up, restated for a check
    import math

    r = int((1.0 + math.sqrt(8.0 * qs + 1.0)) * 0.5)
    r = max(r, 1)
    while r * (r - 1) // 2 > qs:
        r -= 1
    while (r + 1) * r // 2 <= qs:
        r += 1
    return r, qs - r * (r - 1) // 2


def test_triangular_root_against_bisection():
    rng = np.random.default_rng(0)
    qs = list(rng.integers(0, 2 ** 50, size=2000)) + [0, 1, 2, 3, 2 ** 40, 1439302457279]
    for q in qs:
        q = int(q)
        i, j = pair_from_index(q)
        lo, hi = 1, 2 ** 27
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if mid * (mid - 1) // 2 <= q:
                lo = mid
            else:
                hi = mid - 1
        assert (i, j) == (lo, q - lo * (lo - 1) // 2)
        assert 0 <= j < i
