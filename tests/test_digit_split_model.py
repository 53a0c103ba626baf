"""CPU model of the exact digit split behind the tensor-core forms.

Readings 20 to 22 claim that rounding each value to 2^-56 of a power-of-two
scale (per Gram column, or per row of Y and per column of R_JK in the
substitution; the scale more than twice the largest value) and cutting it into
eight signed digits in [-64, 64] (the balanced split) makes every digit
product and every tile sum exact in FP32, and that a product of k terms
through the split differs from the exact one by less than
    2^-57 (sigma ||r||_1 + tau ||y||_1) + k 2^-55 sigma tau + 2^-56 sigma tau:
rounding each value to half a unit of 2^-56 of its scale, the digit pairs
with s + t >= 8 that are not formed (at most 7 * 64^2 * 2^-70 of sigma tau per
term), and the fold's final truncation. The rounding and the signed digits
make the error zero-mean; the truncating split it replaces biased every |x|
low, so Gram diagonals came out low on average. These tests check those
claims with exact integer arithmetic (Python ints), independent of any GPU
code: the bounds on the tile sums that the kernels rely on (worst case, all
digits at their largest magnitude), the fold W = 2^21 U + floor(T / 2^7), the
error bound on random, badly scaled and worst-case inputs, and the absence of
bias.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

DIGITS, BITS = 8, 7
BIAS56 = sum(64 << (7 * s) for s in range(DIGITS))  # 64 in every 7-bit field


def scale_exp(vals):
    """E with 2^(E-1) > max |v| (the kernels' rule: two above the max's exponent)."""
    mx = max(abs(v) for v in vals)
    if mx == 0:
        return None
    return math.frexp(mx)[1] + 1  # mx < 2^(E-1), mx >= 2^(E-2)


def round_half_away(q):
    """Nearest integer to the Fraction q, half-way cases away from zero."""
    a = abs(q)
    n = math.floor(a + Fraction(1, 2))
    return n if q >= 0 else -n


def digits(v, E):
    """Signed digits d_0 .. d_7 of v relative to 2^E: N = round(v 2^(56-E)),
    M = N + BIAS56, d_s = field s of M less 64 (field 0: the bits above 49)."""
    N = round_half_away(Fraction(v) * Fraction(2) ** (56 - E))
    assert abs(N) < 2 ** 55
    M = N + BIAS56
    assert 0 <= M < 129 * 2 ** 49
    ds = [(M >> 49) - 64] + [((M >> (49 - 7 * s)) & 127) - 64 for s in range(1, DIGITS)]
    assert sum(d << (7 * (DIGITS - 1 - s)) for s, d in enumerate(ds)) == N
    return ds


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


def test_digits_represent_values_to_2_pow_minus_57():
    rng = np.random.default_rng(11)
    for _ in range(2000):
        v = float(rng.standard_normal() * 10.0 ** rng.integers(-30, 30))
        E = scale_exp([v, v * 0.5])
        ds = digits(v, E)
        err = abs(value_of(ds, E) - Fraction(v))
        assert err <= Fraction(2) ** (E - 57)
        assert all(-64 <= d <= 63 for d in ds[1:]) and -64 <= ds[0] <= 64


def test_digit_extremes():
    """The largest value below the scale's half gives the top digit 64, the
    most negative -64; a BF16 number represents every digit exactly."""
    E = 1
    top = 1.0 - 2.0 ** -53  # < 2^(E-1) = 1
    assert digits(top, E)[0] == 64 and digits(-top, E)[0] == -64
    for d in range(-64, 65):
        assert float(np.float32(d)) == d and (abs(d) < 256)  # 8 significant bits suffice


@pytest.mark.parametrize("k,rows_per_tile", [(16, 1), (32, 1), (64, 1024)])
def test_worst_case_tile_sums_within_2_pow_24(k, rows_per_tile):
    """All digits at magnitude 64 (the bound): the substitution's tiles (k = 16,
    32 per entry) stay below 2^22 (the kernels' float-to-integer step needs
    that), and the Gram's tiles (64-row chunks read back every 1024 rows, at
    most 4 pairs per tile in each lane half) stay within 2^24, exact in FP32."""
    if rows_per_tile == 1:
        worst = max((e + 1) * k * 64 * 64 for e in range(DIGITS))
        assert worst < 2 ** 22
    else:
        worst = 4 * rows_per_tile * 64 * 64  # lane-half pairing of the Gram kernel
    assert worst <= 2 ** 24


def test_fold_bounds_fit_int64():
    k = 32
    D = [(e + 1) * k * 64 * 64 for e in range(DIGITS)]
    U = sum(D[e] * 2 ** (7 * (3 - e)) for e in range(4))
    T = sum(D[e] * 2 ** (7 * (7 - e)) for e in range(4, 8))
    assert U < 2 ** 41.1 and T < 2 ** 43.4
    assert abs(fold(D)) < 2 ** 62.2 and abs(fold([-d for d in D])) < 2 ** 62.2 + 1
    # the Gram's per-group sums: 4 pairs of 1024 rows per tile half
    G = 4 * 1024 * 64 * 64
    assert G * sum(2 ** (7 * (3 - e)) for e in range(4)) < 2 ** 45.1


def split_bound(y, r, Ey, Er):
    sig, tau = Fraction(2) ** Ey, Fraction(2) ** Er
    return (Fraction(2) ** -57 * (sig * sum(Fraction(abs(float(b))) for b in r)
                                 + tau * sum(Fraction(abs(float(a))) for a in y))
            + (len(y) * Fraction(2) ** -55 + Fraction(2) ** -56) * sig * tau)


@pytest.mark.parametrize("k", [16, 32])
def test_product_error_within_stated_bound(k):
    """|model - exact| <= 2^-57 (sigma ||r||_1 + tau ||y||_1) + (k 2^-55 +
    2^-56) sigma tau, with sigma, tau the power-of-two scales, on random and
    badly scaled vectors; in norm terms at most about 4 k u ||y||_2 ||r||_2,
    the order of the FP64 dot product's gamma_k bound."""
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
    """Values whose digits 1..7 are all -64 (N = 64 2^49 - 64 (2^49 - 1) / 127 * 127 ...,
    chosen digit by digit): the pairs that are not formed then add up with one
    sign, and the error comes within a factor 4 of the bound's k 2^-55 sigma tau
    term, so that term is needed and not loose."""
    E = 1
    ds = [64] + [-64] * 7
    N = sum(d << (7 * (DIGITS - 1 - s)) for s, d in enumerate(ds))
    v = float(Fraction(N) * Fraction(2) ** (E - 56))
    assert digits(v, E) == ds
    y, r = [v] * k, [v] * k
    got, Ey, Er, Dmax = model_dot(y, r)
    assert Ey == E and Er == E and Dmax <= 2 ** 22
    exact = sum(Fraction(a) * Fraction(b) for a, b in zip(y, r))
    err = abs(got - exact)
    assert err <= split_bound(y, r, Ey, Er)
    assert err >= k * Fraction(2) ** -55 * Fraction(2) ** (Ey + Er) / 4


def gram_diag_model(q):
    """A Gram diagonal q . q as the Gram kernel forms it: the tile sums of the
    pairs s + t <= 7, plus the square pair (4, 4) of e = 8, sum_i d_4(q_i)^2,
    which the kernel accumulates exactly on the side (weight 2^-70 of
    sigma^2). The other dropped pairs of a square are products of different
    digits (zero mean) or squares 2^-14 smaller."""
    got, E, _, _ = model_dot(q, q)
    if E is None:
        return got, E
    s44 = sum(digits(v, E)[4] ** 2 for v in q)
    return got + Fraction(s44) * Fraction(2) ** (2 * E - 70), E


def test_gram_diagonal_is_unbiased():
    """Reading 22: the truncating split lowered Gram diagonals by about 3.7 u
    relative on average. With the balanced split alone, the dropped square
    pair (4, 4) still lowers them (about -0.7 u here, more where the column
    scale is far above the typical value); with its exact sum added, the mean
    error is zero to within sampling noise (below 0.1 u here)."""
    rng = np.random.default_rng(22)
    errs, errs_plain = [], []
    for _ in range(40):
        q = list(map(float, rng.standard_normal(256)))
        exact = sum(Fraction(a) * Fraction(a) for a in q)
        got, _ = gram_diag_model(q)
        plain, _, _, _ = model_dot(q, q)
        errs.append(float((got - exact) / exact))
        errs_plain.append(float((plain - exact) / exact))
    u = 2.0 ** -53
    assert np.mean(errs_plain) < -0.3 * u  # the bias the side sum removes
    assert abs(np.mean(errs)) < 0.1 * u, (np.mean(errs) / u)


def test_off_diagonal_products_are_unbiased():
    """Products of different values (Gram off-diagonals, the substitution's
    y_J R_JK) have zero-mean error without any correction."""
    rng = np.random.default_rng(23)
    errs = []
    for _ in range(60):
        y = list(map(float, rng.standard_normal(32)))
        r = list(map(float, rng.standard_normal(32)))
        got, _, _, _ = model_dot(y, r)
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(y, r))
        errs.append(float(got - exact) / float(np.linalg.norm(y) * np.linalg.norm(r)))
    u = 2.0 ** -53
    assert abs(np.mean(errs)) < 0.2 * u, (np.mean(errs) / u)


def test_gram_entry_error_matches_norm_wise_bound():
    """A Gram entry of m rows through the split (scale per column) differs
    from q_j . q_k by at most m 2^-54 sigma_j sigma_k (the bound above with
    k = m; the rounding terms are below m 2^-56 sigma_j sigma_k): with
    sigma <= 4 max |q| this is at most about 8.5 m u ||q_j|| ||q_k||, so
    ||E|| <= 8.5 m n u ||Q||^2, inside the 11 (mn + n(n+1)) u ||Q||^2 shift of
    Eq. (finds2)."""
    rng = np.random.default_rng(7)
    m = 300
    for _ in range(20):
        qj = rng.standard_normal(m) * 10.0 ** rng.integers(-5, 5)
        qk = rng.standard_normal(m) * 10.0 ** rng.integers(-5, 5)
        got, Ej, Ek, Dmax = model_dot(list(map(float, qj)), list(map(float, qk)))
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(qj, qk))
        assert abs(got - exact) <= m * Fraction(2) ** -54 * Fraction(2) ** (Ej + Ek)


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


def test_fixed_point_shift_form():
    """The kernels form N = round(x 2^(56-E)) from the bit pattern as
    (4 mant + 2^(K-1)) >> K with K = 1021 + E - ex capped to [0, 63] (mant the
    53-bit significand, ex the biased exponent): the same integer as rounding
    half away from zero, for normal and subnormal x and every scale the
    kernels' rule gives (|x| < 2^(E-1))."""
    rng = np.random.default_rng(21)
    vals = [float(v) for v in rng.standard_normal(3000) * 10.0 ** rng.integers(-300, 300, 3000)]
    vals += [5e-324, 2.2250738585072014e-308, 1.0 - 2.0 ** -53, 0.75, 2.0 ** -1074 * 3]
    for v in vals:
        if v == 0.0 or not math.isfinite(v):
            continue
        bits = int(np.float64(abs(v)).view(np.uint64))
        for extra in (0, 1, 2, 40, 80):
            # the kernels' scale rule: (exponent field, 1 for subnormals) - 1021,
            # which keeps K >= 0 for subnormal values as well
            E = max((bits >> 52) & 0x7FF, 1) - 1021 + extra  # |v| < 2^(E-1)
            ex = (bits >> 52) & 0x7FF
            mant = bits & ((1 << 52) - 1)
            if ex:
                mant |= 1 << 52
            else:
                ex = 1
            K = min(max(1021 + E - ex, 0), 63)
            N = ((mant << 2) + ((1 << K) >> 1)) >> K
            assert N == abs(round_half_away(Fraction(v) * Fraction(2) ** (56 - E))), (v, E)


def test_digit_fields_from_14_bit_chunks():
    """The kernels take the 7-bit fields two at a time: chunk j = bits
    42 - 14 j up of M (two values side by side in one 32-bit word, low 16 bits
    each), field 2 j = (chunk >> 7) & 127 (& 255 for j = 0: the top field
    holds up to 128), field 2 j + 1 = chunk & 127; the same fields as
    (M >> (49 - 7 s)) & 127."""
    rng = np.random.default_rng(22)
    for _ in range(3000):
        N = int(rng.integers(-(2 ** 55) + 1, 2 ** 55))
        M0 = N + BIAS56
        M1 = int(rng.integers(-(2 ** 55) + 1, 2 ** 55)) + BIAS56
        for j in range(4):
            t0 = (M0 >> (42 - 14 * j)) & 0xFFFFFFFF
            t1 = (M1 >> (42 - 14 * j)) & 0xFFFFFFFF
            C = (t0 & 0xFFFF) | ((t1 & 0xFFFF) << 16)  # byte_perm(t0, t1, 0x5410)
            ev = (C >> 7) & (0x00FF00FF if j == 0 else 0x007F007F)
            od = C & 0x007F007F
            for M, sh in ((M0, 0), (M1, 16)):
                f_even = (M >> 49) if j == 0 else (M >> (49 - 7 * (2 * j))) & 127
                f_odd = (M >> (49 - 7 * (2 * j + 1))) & 127
                assert (ev >> sh) & 0xFFFF == f_even and (od >> sh) & 0xFFFF == f_odd


def test_pairwise_fold_in_32_bits():
    """The one-sweep substitution and the update kernel (K <= 32: at most 8
    digit pairs x 32 columns x 64^2 per tile) fold tile sums |D_e| <= 2^20 as
    b_e = 0x4B400000 + D_e (the float bits of D_e + 1.5 2^23), pairs
    P = b_e 2^7 + b_(e+1) - 129 * 0x4B400000 in 32-bit wrap-around arithmetic
    (the true value below 2^28), and W = P01 2^35 + P23 2^21 + P45 2^7 +
    floor(P67 / 2^7): the same W as the int64 fold."""
    rng = np.random.default_rng(23)
    C129 = (0x4B400000 * 129) & 0xFFFFFFFF
    cases = [[2 ** 20] * 8, [-(2 ** 20)] * 8, [0] * 8, [2 ** 20, -(2 ** 20)] * 4]
    cases += [list(rng.integers(-(2 ** 20), 2 ** 20 + 1, 8)) for _ in range(5000)]
    for D in cases:
        D = [int(d) for d in D]
        assert float(np.float32(D[0] + 1.5 * 2 ** 23)) == D[0] + 1.5 * 2 ** 23
        b = [(0x4B400000 + d) & 0xFFFFFFFF for d in D]

        def pair(x, y):
            p = (x * 128 + y - C129) & 0xFFFFFFFF
            return p - (1 << 32) if p >= 1 << 31 else p

        p01, p23, p45, p67 = pair(b[0], b[1]), pair(b[2], b[3]), pair(b[4], b[5]), pair(b[6], b[7])
        assert p01 == D[0] * 128 + D[1] and abs(p01) < 2 ** 28
        W = (p01 << 35) + (p23 << 21) + (p45 << 7) + (p67 >> 7)
        assert W == fold(D) and abs(W) < 2 ** 63


def test_gram_mma_program_covers_each_pair_once():
    """The Gram kernel's six MMAs per K step: A = digit planes s (lanes 0..63)
    and s + 1 (lanes 64..127), B = planes t0 .. t0 + nt - 1 side by side, from
    tensor column 64 (s + t0). The read-back takes d = x from lanes 0..63 of
    tile x and d = x + 1 from lanes 64..127 of tiles 0..6. Every pair with
    s + t <= 7 lands in exactly one cell that is read, with d = s + t; each
    lane half of a tile holds at most 4 pairs (the 2^24 bound); the columns
    stay within the 512 of tensor memory; N <= 256 per MMA."""
    program = [(0, 0, 4), (0, 4, 4), (2, 0, 4), (2, 4, 2), (4, 0, 4), (6, 0, 2)]
    cells = {}
    for s, t0, nt in program:
        assert 64 * (s + t0) + 64 * nt <= 512 and 64 * nt <= 256
        for i in range(nt):
            t = t0 + i
            tile = s + t
            cells.setdefault((tile, "lo"), []).append((s, t))
            cells.setdefault((tile, "hi"), []).append((s + 1, t))
    read = {}
    for (tile, half), pairs in cells.items():
        assert len(pairs) <= 4
        d = tile if half == "lo" else tile + 1
        if d > 7:
            continue  # never read back
        for s, t in pairs:
            assert s + t == d
            read[(s, t)] = read.get((s, t), 0) + 1
    want = {(s, t) for s in range(8) for t in range(8) if s + t <= 7}
    assert set(read) == want and all(c == 1 for c in read.values())
    # the bench's flop count: N adds up to 1280 per K step
    assert sum(64 * nt for _, _, nt in program) == 1280


def test_gram_group_value_fits_and_rounds():
    """Per 1024-row group the Gram kernel folds its exact digit sums into
    U = sum_{d<=3} D_d 2^(7(3-d)) and T = sum_{d>=4} D_d 2^(7(7-d)) (|D_d| <=
    4 * 1024 * 64^2 = 2^24 per share) and converts W = 2^17 U + round(T / 2^11)
    to FP64: W stays below 2^62.2 (int64), and W 2^-52 differs from
    2^-35 U + 2^-63 T by at most 2^-53 (in units of sigma_j sigma_k)."""
    G = 4 * 1024 * 64 * 64
    rng = np.random.default_rng(24)
    cases = [[G] * 8, [-G] * 8, [G, -G] * 4] + [list(rng.integers(-G, G + 1, 8)) for _ in range(3000)]
    for D in cases:
        D = [int(d) for d in D]
        U = sum(D[e] * 2 ** (7 * (3 - e)) for e in range(4))
        T = sum(D[e] * 2 ** (7 * (7 - e)) for e in range(4, 8))
        assert abs(U) < 2 ** 45.1 and abs(T) < 2 ** 45.1
        W = (U << 17) + ((T + 1024) >> 11)
        assert abs(W) < 2 ** 62.2
        exact = Fraction(U, 2 ** 35) + Fraction(T, 2 ** 63)
        assert abs(Fraction(W, 2 ** 52) - exact) <= Fraction(1, 2 ** 53)


def model_dot7(y, r):
    """y . r as the adjoint's product kernel forms it: the seven leading digits
    of each value, tile sums over the pairs s + t <= 6, W = sum_e D_e 2^(42 - 7e),
    value 2^(Ey + Er - 56) W."""
    Ey, Er = scale_exp(y), scale_exp(r)
    if Ey is None or Er is None:
        return Fraction(0), None, None, 0, 0
    ya = [digits(v, Ey)[:7] for v in y]
    rb = [digits(v, Er)[:7] for v in r]
    D = [0] * 7
    for a, b in zip(ya, rb):
        for s in range(7):
            for t in range(7 - s):
                D[s + t] += a[s] * b[t]
    W = sum(D[e] << (42 - 7 * e) for e in range(7))
    return Fraction(W) * Fraction(2) ** (Ey + Er - 56), Ey, Er, max(abs(d) for d in D), W


def test_seven_digit_products_of_the_adjoint_kernel():
    """The adjoint's product kernel (K = 64, seven digits per value): every tile
    sum below 2^21 (exact in FP32, and D_e + 1.5 2^23 exact), W below 2^61, and
    the product within 2^-49 (sigma ||r||_1 + tau ||y||_1) + 64 * 7 * 2^-51
    sigma tau of the exact dot product, on random, badly scaled and worst-case
    vectors; the pairwise 32-bit fold gives the same W."""
    k = 64
    rng = np.random.default_rng(64)
    C129 = (0x4B400000 * 129) & 0xFFFFFFFF

    def pair(x, y):
        p = (x * 128 + y - C129) & 0xFFFFFFFF
        return p - (1 << 32) if p >= 1 << 31 else p

    E = 1
    worst = float(Fraction(sum(d << (7 * (DIGITS - 1 - s)) for s, d in enumerate([64] + [-64] * 7)))
                  * Fraction(2) ** (E - 56))
    cases = [([worst] * k, [worst] * k)]
    for trial in range(120):
        y = rng.standard_normal(k) * np.exp2(rng.integers(-40, 40, size=k) * (trial % 3 == 0))
        r = rng.standard_normal(k) * np.exp2(rng.integers(-40, 40, size=k) * (trial % 4 == 0))
        cases.append((list(map(float, y)), list(map(float, r))))
    for y, r in cases:
        got, Ey, Er, Dmax, W = model_dot7(y, r)
        assert Dmax < 2 ** 21 and abs(W) < 2 ** 61
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(y, r))
        sig, tau = Fraction(2) ** Ey, Fraction(2) ** Er
        bound = (Fraction(2) ** -49 * (sig * sum(Fraction(abs(b)) for b in r) + tau * sum(Fraction(abs(a)) for a in y))
                 + 64 * 7 * Fraction(2) ** -51 * sig * tau)
        assert abs(got - exact) <= bound
        # the kernel's fold: b_e = 0x4B400000 + D_e, pairs in 32 bits, D_6 alone
        ya = [digits(v, Ey)[:7] for v in y]
        rb = [digits(v, Er)[:7] for v in r]
        D = [sum(a[s] * b[e - s] for a, b in zip(ya, rb) for s in range(e + 1)) for e in range(7)]
        bb = [(0x4B400000 + d) & 0xFFFFFFFF for d in D]
        d6 = bb[6] - 0x4B400000
        assert (pair(bb[0], bb[1]) << 35) + (pair(bb[2], bb[3]) << 21) + (pair(bb[4], bb[5]) << 7) + d6 == W


def test_adjoint_product_mma_program():
    """Group g's MMAs: digit s (A) against the planes t = 0 .. 6 - s of the
    group side by side (N = 32 (7 - s)) from accumulator column 32 s; plane t
    then lands in columns 32 (s + t) .. +31, tile e = s + t. Every pair with
    s + t <= 6 is formed once per K step, the first MMA (s = 0) covers all 7
    tiles, and the 7 tiles fit one 256-column accumulator (two in 512). For
    the columns 0..31 of Q_{k-1} = Q_k R_k only the K steps 0, 1 (rows 0..31 of
    R_k) can be non-zero: R_k is upper triangular."""
    seen = {}
    for s in range(7):
        N = 32 * (7 - s)
        assert N % 16 == 0 and 16 <= N <= 256
        for t in range(N // 32):
            col = 32 * s + 32 * t
            assert col + 32 <= 224
            seen[(s, t)] = col // 32
    assert sorted(seen) == [(s, t) for s in range(7) for t in range(7) if s + t <= 6]
    assert all(e == s + t for (s, t), e in seen.items())
    R = np.triu(np.ones((64, 64)))
    assert not R[32:, :32].any()
