"""CPU model of the exact digit split behind the tensor-core forms.

Readings 20 and 21 claim that cutting each value into eight signed 7-bit
digits relative to a power-of-two scale (per Gram column, or per row of Y and
per column of R_JK in the substitution) makes every digit product and every
tile sum exact in FP32, and that a product of k terms through the split
differs from the exact one by less than
    2^-56 (sigma ||r||_1 + tau ||y||_1) + k 2^-53 sigma tau:
truncating each value to 2^-56 of its scale, plus the digit pairs with
s + t >= 8 that are not formed (at most 7 127^2 2^-70 < 2^-53.2 of sigma tau
per term). These tests check those claims with exact integer arithmetic
(Python ints), independent of any GPU code: the bounds on the tile sums that
the kernels rely on (worst case, all digits 127), the fold
W = 2^21 U + floor(T / 2^7), and the error bound on random, badly scaled and
worst-case inputs.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

DIGITS, BITS = 8, 7


def scale_exp(vals):
    """E with 2^E > max |v| (the kernels' rule: one above the max's exponent)."""
    mx = max(abs(v) for v in vals)
    if mx == 0:
        return None
    return math.frexp(mx)[1]  # mx < 2^E, mx >= 2^(E-1)


def digits(v, E):
    """Signed 7-bit digits a_0 .. a_7 of v relative to 2^E: F = floor(|v| 2^(56-E))."""
    F = math.floor(Fraction(abs(v)) * Fraction(2) ** (56 - E))
    assert F < 2 ** 56
    sgn = -1 if v < 0 else 1
    return [sgn * ((F >> (49 - 7 * s)) & 127) for s in range(DIGITS)]


def value_of(ds, E):
    return sum(Fraction(d) * Fraction(2) ** (E - 7 * (s + 1)) for s, d in enumerate(ds))


def tile_sums(ya, rb):
    """D_e = sum over k and pairs (s, t) with s + t = e of a_s b_t (e = 0 .. 7)."""
    D = [0] * DIGITS
    for a, b in zip(ya, rb):
        for s in range(DIGITS):
            for t in range(DIGITS - s):
                D[s + t] += a[s] * b[t]
    return D


def fold(D):
    U = D[0] * 2 ** 21 + D[1] * 2 ** 14 + D[2] * 2 ** 7 + D[3]
    T = D[4] * 2 ** 21 + D[5] * 2 ** 14 + D[6] * 2 ** 7 + D[7]
    return (U << 21) + (T >> 7)  # Python >> floors, like the kernels' arithmetic shift


def model_dot(y, r):
    """y . r through the split: scale per vector, digits, tile sums, fold."""
    Ey, Er = scale_exp(y), scale_exp(r)
    if Ey is None or Er is None:
        return Fraction(0), None, None, 0
    ya = [digits(v, Ey) for v in y]
    rb = [digits(v, Er) for v in r]
    D = tile_sums(ya, rb)
    W = fold(D)
    return Fraction(W) * Fraction(2) ** (Ey + Er - 56), Ey, Er, max(abs(d) for d in D)


def test_digits_represent_values_to_2_pow_minus_56():
    rng = np.random.default_rng(11)
    for _ in range(2000):
        v = float(rng.standard_normal() * 10.0 ** rng.integers(-30, 30))
        E = scale_exp([v, v * 0.5])
        err = abs(value_of(digits(v, E), E) - Fraction(v))
        assert err < Fraction(2) ** (E - 56)
        assert all(abs(d) <= 127 for d in digits(v, E))


@pytest.mark.parametrize("k,rows_per_tile", [(16, 1), (32, 1), (64, 256)])
def test_worst_case_tile_sums_below_2_pow_24(k, rows_per_tile):
    """All digits at 127 (the bound): the substitution's tiles (k = 16, 32 per
    entry) and the Gram's tiles (64-row chunks read back every 256 rows, at
    most 4 pairs per tile in each lane half) stay exact in FP32."""
    if rows_per_tile == 1:
        worst = max((e + 1) * k * 127 * 127 for e in range(DIGITS))
    else:
        worst = 4 * rows_per_tile * 127 * 127  # lane-half pairing of the Gram kernel
    assert worst < 2 ** 24


def test_fold_bounds_fit_int64():
    k = 32
    D = [(e + 1) * k * 127 * 127 for e in range(DIGITS)]
    U = sum(D[e] * 2 ** (7 * (3 - e)) for e in range(4))
    T = sum(D[e] * 2 ** (7 * (7 - e)) for e in range(4, 8))
    assert U < 2 ** 40.1 and T < 2 ** 42.4
    assert abs(fold(D)) < 2 ** 61.2 and abs(fold([-d for d in D])) < 2 ** 61.2 + 1


def split_bound(y, r, Ey, Er):
    sig, tau = Fraction(2) ** Ey, Fraction(2) ** Er
    return (Fraction(2) ** -56 * (sig * sum(Fraction(abs(float(b))) for b in r)
                                 + tau * sum(Fraction(abs(float(a))) for a in y))
            + len(y) * Fraction(2) ** -53 * sig * tau)


@pytest.mark.parametrize("k", [16, 32])
def test_product_error_within_stated_bound(k):
    """|model - exact| <= 2^-56 (sigma ||r||_1 + tau ||y||_1) + k 2^-53 sigma
    tau, with sigma, tau the power-of-two scales, on random and badly scaled
    vectors; in norm terms at most about 4 k u ||y||_2 ||r||_2, the order of
    the FP64 dot product's gamma_k bound."""
    rng = np.random.default_rng(100 + k)
    for trial in range(300):
        y = rng.standard_normal(k) * np.exp2(rng.integers(-40, 40, size=k) * (trial % 3 == 0))
        r = rng.standard_normal(k) * np.exp2(rng.integers(-40, 40, size=k) * (trial % 5 == 0))
        if trial % 7 == 0:
            y[rng.integers(k)] = 0.0
        y, r = list(map(float, y)), list(map(float, r))
        got, Ey, Er, _ = model_dot(y, r)
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(y, r))
        err = abs(got - exact)
        assert err <= split_bound(y, r, Ey, Er), (trial, float(err), float(split_bound(y, r, Ey, Er)))
        u = Fraction(2) ** -53
        assert err <= 4 * k * u * Fraction(np.linalg.norm(y)) * Fraction(np.linalg.norm(r)) * Fraction(1.001)


@pytest.mark.parametrize("k", [16, 32])
def test_worst_case_dropped_pairs_near_the_bound(k):
    """Every value at the top of its scale (F = 2^56 - 8: every digit 127 but
    the last, 120):
    the digit pairs that are not formed make the largest error, and it comes
    within a factor 2 of the bound's k 2^-53 sigma tau term, so that term is
    needed and not loose."""
    v = 1.0 - 2.0 ** -53  # scale 2^0 > v
    y, r = [v] * k, [v] * k
    got, Ey, Er, Dmax = model_dot(y, r)
    assert Ey == 0 and Er == 0 and Dmax < 2 ** 24
    exact = sum(Fraction(a) * Fraction(b) for a, b in zip(y, r))
    err = abs(got - exact)
    assert err <= split_bound(y, r, Ey, Er)
    assert err >= k * Fraction(2) ** -53 * Fraction(1, 2)


def test_gram_entry_error_matches_norm_wise_bound():
    """A Gram entry of m rows through the split (scale per column) differs
    from q_j . q_k by at most m 2^-53 sigma_j sigma_k (the bound above with
    k = m; the truncation terms are below m 2^-55 sigma_j sigma_k): with
    sigma <= 2 max |q| this is at most about 4.3 m u ||q_j|| ||q_k||, so
    ||E|| <= 4.3 m n u ||Q||^2, inside the 11 (mn + n(n+1)) u ||Q||^2 shift of
    Eq. (finds2)."""
    rng = np.random.default_rng(7)
    m = 300
    for _ in range(20):
        qj = rng.standard_normal(m) * 10.0 ** rng.integers(-5, 5)
        qk = rng.standard_normal(m) * 10.0 ** rng.integers(-5, 5)
        got, Ej, Ek, Dmax = model_dot(list(map(float, qj)), list(map(float, qk)))
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(qj, qk))
        assert abs(got - exact) <= m * Fraction(2) ** -53 * Fraction(2) ** (Ej + Ek)


def test_exact_for_short_integers():
    """Values with few significant bits relative to the scale are represented
    exactly, so their products come out exact."""
    y = [3.0, -5.0, 7.0, 1.0] * 4
    r = [2.0, 4.0, -6.0, 8.0] * 4
    got, _, _, _ = model_dot(y, r)
    assert got == sum(Fraction(a) * Fraction(b) for a, b in zip(y, r))


def _solve_fp64(x, R, cols):
    """Forward substitution of y R = x on the given columns, FP64, multiplying
    by the rounded reciprocal of r_jj as the GPU's pass kernel does."""
    for j in cols:
        t = x[j]
        for i in cols:
            if i >= j:
                break
            t = t - x[i] * R[i, j]
        x[j] = t * (1.0 / R[j, j])


@pytest.mark.parametrize("n,w,kappa", [(64, 16, 10.0), (64, 32, 1e3), (100, 32, 30.0), (128, 32, 1e2)])
def test_blocked_substitution_backward_error(n, w, kappa):
    """Reading 21: the substitution in w-column blocks, with y_J R_JK through the
    split and the diagonal blocks in FP64, keeps the row-wise backward error of
    Eq. (backward2), ||x - y R|| / (||y|| ||R||) = O(u): within 4 n u, and
    within a small factor of plain FP64 substitution on the same rows (seen:
    1.2 to 4.5 times, both near 1e-16). R is moderately conditioned so that
    ||y|| ||R|| is of the order of ||x|| and the measure resolves rounding."""
    rng = np.random.default_rng(n + w)
    Qa, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Qb, _ = np.linalg.qr(rng.standard_normal((n, n)))
    R = np.linalg.qr(Qa @ np.diag(np.geomspace(1.0, 1.0 / kappa, n)) @ Qb, mode="r")
    R = R * np.sign(np.diag(R))[:, None]
    u = 2.0 ** -53
    normR = np.linalg.norm(R, 2)
    for trial in range(6):
        x0 = rng.standard_normal(n) * np.exp2(rng.integers(-5, 5, size=n))
        # blocked: FP64 diagonal blocks, split-model off-diagonal products
        y = x0.copy()
        for J in range(0, n, w):
            _solve_fp64(y, R, list(range(J, min(J + w, n))))
            yJ = [float(v) for v in y[J:J + w]]
            for c in range(J + w, n):
                prod, _, _, _ = model_dot(yJ, [float(v) for v in R[J:J + w, c]])
                y[c] = y[c] - float(prod)
        # plain FP64 substitution of the same row
        z = x0.copy()
        _solve_fp64(z, R, list(range(n)))
        eb = np.linalg.norm(x0 - y @ R) / (np.linalg.norm(y) * normR)
        ez = np.linalg.norm(x0 - z @ R) / (np.linalg.norm(z) * normR)
        assert eb <= 4 * n * u and ez <= 4 * n * u, (trial, eb, ez)
        assert eb <= 16 * max(ez, u), (trial, eb, ez)
