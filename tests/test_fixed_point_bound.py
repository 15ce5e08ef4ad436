"""The arithmetic of the exact fixed-point X passes (FP64 block utilities),
restated on the host with Python integers and checked against exact rational
arithmetic: a lane's vector z is scaled to z_fx = round(z 2^k) with
|z_fx| <= 2^(62 - bx) (k from max|z|), split into halves hi 2^31 + lo
(0 <= lo < 2^31), the products x_int lo and x_int hi are summed separately in
64-bit integers and combined; the result, rounded once to FP64, differs from
the exact sum_j x_ij z_j by at most 2^(bx - 63) max|z| sum_j |x_ij| (the
rounding of z to 2^-k) plus one FP64 rounding of the result.  This pins the
bound the design states, and that neither partial sum leaves 64 bits for sums
of fewer than 2^(32 - bx) terms.  The kernels themselves are checked against
the oracle on the GPU (test_gpu_exact_passes.py)."""
import math
from fractions import Fraction

import numpy as np
import pytest


def _scale_exponent(zmax: float, bx: int) -> int:
    _, e = math.frexp(zmax)          # zmax < 2^e
    return 62 - bx - e


def _fixed_sum(x_int, z, bx):
    k = _scale_exponent(max(abs(v) for v in z), bx)
    lo_sum = hi_sum = 0
    for xi, zj in zip(x_int, z):
        q = round(math.ldexp(zj, k))                     # round half to even, as llrint
        assert abs(q) <= 2 ** (62 - bx)
        hi, lo = q >> 31, q & (2 ** 31 - 1)
        assert 0 <= lo < 2 ** 31 and abs(hi) <= 2 ** (31 - bx)
        lo_sum += xi * lo
        hi_sum += xi * hi
        assert abs(lo_sum) < 2 ** 63 and abs(hi_sum) < 2 ** 63   # the two 64-bit sums
    total = (hi_sum << 31) + lo_sum                       # exact, 128-bit
    return float(Fraction(total, 2 ** k)), k


@pytest.mark.parametrize("bx,sx", [(1, 0), (4, 0), (5, 2), (10, 0)])
@pytest.mark.parametrize("spread", [0.0, 6.0, 12.0])
def test_fixed_point_sum_within_bound(bx, sx, spread):
    rng = np.random.default_rng(100 * bx + int(spread))
    for trial in range(40):
        m = int(rng.integers(1, 400))
        mag = 2 ** (bx - 1)
        x_int = [int(v) for v in rng.integers(-mag, mag, m)] if bx > 1 else [1] * m
        x_int = [v if v != 0 else 1 for v in x_int]
        z = list(rng.standard_normal(m) * 10.0 ** rng.uniform(-spread, spread, m))
        got, k = _fixed_sum(x_int, z, bx)
        # exact value of sum x_ij z_j, x = x_int 2^-sx (the scale 2^-sx is exact)
        exact = sum(Fraction(xi) * Fraction(zj) for xi, zj in zip(x_int, z))
        got_x = math.ldexp(got, -sx)
        exact_x = exact / 2 ** sx
        zmax = max(abs(v) for v in z)
        bound = Fraction(2) ** (bx - 63) * Fraction(zmax) * sum(abs(Fraction(v)) for v in x_int) / 2 ** sx
        err = abs(Fraction(got_x) - exact_x)
        assert err <= bound + abs(exact_x) * Fraction(2) ** -52, (trial, float(err), float(bound))


def test_partial_sums_fit_at_the_term_limit():
    """The longest sums the examination admits: 2^(32 - bx) - 1 terms of the
    largest products stay below 2^63 in both partial sums."""
    for bx in (1, 4, 10):
        terms = 2 ** (32 - bx) - 1
        x_max = 2 ** bx - 1
        assert terms * x_max * (2 ** 31 - 1) < 2 ** 63          # sum of x_int lo
        assert terms * x_max * 2 ** (31 - bx) < 2 ** 63         # sum of x_int hi
