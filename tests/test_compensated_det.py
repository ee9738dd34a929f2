"""The compensated 2x2 determinant the projection uses for the inverse of
the dilated 2D covariance (Sec. 3.3, Sigma' = J W Sigma W^T J^T, its conic
being the inverse): Kahan's scheme with one fused multiply-add to recover
the rounding error of b*b,

    w = fl(b b);  e = fma(-b, b, w);  f = fma(a, c, -w);  det = fl(f + e),

has a relative error of at most 2u in binary32 (u = 2^-24), whatever the
cancellation in a c - b^2 (Jeannerod, Louvet & Muller, "Further analysis of
Kahan's algorithm for the accurate computation of 2x2 determinants", Math.
Comp. 2013).  This CPU test pins that bound for binary32 operands against
exact rational arithmetic on inputs with a c ~ b^2, and shows that the plain
product difference does not meet it there.  CPU only."""
from fractions import Fraction

import numpy as np

U = 2.0 ** -24


def _f32(x) -> np.float32:
    return np.float32(x)


def _fma32(a, b, c) -> np.float32:
    """Correctly rounded binary32 fma: the exact a b + c rounded once (a
    binary32 product is exact in binary64, and the binary64 sum rounded to
    binary32 only differs from one rounding at exact ties, which the exact
    rational check below rules out)."""
    exact = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    r = np.float32(float(exact))
    # Correct the rare double-rounding case by comparing neighbours exactly.
    lo, hi = np.nextafter(r, np.float32(-np.inf)), np.nextafter(r, np.float32(np.inf))
    best = min((lo, r, hi), key=lambda v: abs(Fraction(float(v)) - exact))
    return np.float32(best)


def kahan_det(a, b, c) -> np.float32:
    w = _f32(b * b)
    e = _fma32(-b, b, w)
    f = _fma32(a, c, -w)
    return _f32(f + e)


def naive_det(a, b, c) -> np.float32:
    return _f32(_f32(a * c) - _f32(b * b))


def _ill_conditioned(rng, n):
    """Dilated covariances of needle-thin Gaussians: a long axis of variance
    L, a short one of variance ~0 plus the 0.3 px^2 dilation, rotated."""
    out = []
    for _ in range(n):
        L = 10.0 ** rng.uniform(2, 5)
        th = rng.uniform(0, np.pi)
        cs, sn = np.cos(th), np.sin(th)
        a = _f32(L * cs * cs + 0.3)
        c = _f32(L * sn * sn + 0.3)
        b = _f32(L * cs * sn)
        out.append((a, b, c))
    return out


def test_kahan_determinant_meets_the_2u_bound():
    rng = np.random.default_rng(0)
    worst, worst_naive, n_naive_over = 0.0, 0.0, 0
    for a, b, c in _ill_conditioned(rng, 400):
        exact = Fraction(float(a)) * Fraction(float(c)) - Fraction(float(b)) ** 2
        if exact == 0:
            continue
        k = float(abs((Fraction(float(kahan_det(a, b, c))) - exact) / exact))
        nv = float(abs((Fraction(float(naive_det(a, b, c))) - exact) / exact))
        worst = max(worst, k)
        worst_naive = max(worst_naive, nv)
        n_naive_over += nv > 2 * U
    assert worst <= 2 * U, worst / U
    # The plain difference loses the cancelled digits on these inputs.
    assert worst_naive > 100 * U and n_naive_over > 100


def test_kahan_determinant_exact_cases():
    # Exactly representable products give the exact determinant.
    for a, b, c in [(4.0, 2.0, 1.0), (3.0, 1.0, 5.0), (1e3, 999.0, 998.0)]:
        a, b, c = _f32(a), _f32(b), _f32(c)
        assert Fraction(float(kahan_det(a, b, c))) == Fraction(float(a)) * Fraction(float(c)) - Fraction(float(b)) ** 2
