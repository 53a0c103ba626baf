"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test targets a mistake that could plausibly hide in the oracle (a
dropped term of the shift, a transposed Gram, a wrong TRSM index, a reversed
R accumulation, ...). None of them compares the oracle with itself.
"""
import numpy as np
import pytest

import oracle
from paper_1809_11085_gb300.testmat import (block_diag_spd, dense_spd, geometric_sigma,
                                            repeated_small_sigma, testmat, testmat_factors)

U = 2.0 ** -53


def orth2(Q):
    n = Q.shape[1]
    return np.linalg.norm(Q.T @ Q - np.eye(n), 2)


def resid(X, Q, R):
    return np.linalg.norm(X - Q @ R) / np.linalg.norm(X)


def signfix_qr(Y):
    """Householder QR (LAPACK) with diag(R) > 0: the unique QR factorization."""
    Qh, Rh = np.linalg.qr(Y)
    d = np.sign(np.diag(Rh))
    d[d == 0] = 1.0
    return Qh * d, Rh * d[:, None]


# --------------------------------------------------------------------------- building blocks, exact

def test_gram_exact_on_integers():
    rng = np.random.default_rng(0)
    X = rng.integers(-50, 51, size=(173, 7)).astype(np.float64)
    A = oracle.gram(X)
    Xi = X.astype(np.int64)
    assert np.array_equal(A, (Xi.T @ Xi).astype(np.float64))
    # a non-square, non-symmetric-looking input: X^T X is n x n, not m x m
    assert A.shape == (7, 7)


def test_gram_oblique_exact_on_integers():
    rng = np.random.default_rng(1)
    bs, nb, n = 4, 9, 5
    X = rng.integers(-9, 10, size=(bs * nb, n)).astype(np.float64)
    G = rng.integers(-3, 4, size=(nb, bs, bs))
    Bblk = (np.einsum("kij,kil->kjl", G, G) + np.eye(bs)[None]).astype(np.float64)
    A, fro2 = oracle.gram_oblique(X, Bblk)
    Bfull = np.zeros((bs * nb, bs * nb), dtype=np.int64)
    for k in range(nb):
        Bfull[k * bs:(k + 1) * bs, k * bs:(k + 1) * bs] = Bblk[k].astype(np.int64)
    Xi = X.astype(np.int64)
    assert np.array_equal(A, (Xi.T @ Bfull @ Xi).astype(np.float64))
    assert fro2 == float((Xi * Xi).sum())


def _int_upper(n, rng, diag=(1.0, 2.0, 4.0)):
    """Upper triangular with power-of-two diagonal: substitution and Cholesky are exact."""
    R = np.triu(rng.integers(-4, 5, size=(n, n))).astype(np.float64)
    R[np.diag_indices(n)] = rng.choice(diag, size=n)
    return R


def test_chol_exact_and_shift_added_to_diagonal():
    rng = np.random.default_rng(2)
    for n in (1, 2, 5, 11):
        R = _int_upper(n, rng)
        A = R.T @ R
        Rc, fail = oracle.chol(A)
        assert fail == 0 and np.array_equal(Rc, R)
        # chol(A' + sI) with A' = A - sI must give back R: the shift goes on the diagonal
        Rc2, fail2 = oracle.chol(A - 0.5 * np.eye(n), 0.5)
        assert fail2 == 0 and np.array_equal(Rc2, R)
        assert np.array_equal(np.tril(Rc, -1), np.zeros((n, n)))


def test_chol_breakdown_column():
    A = np.diag([4.0, 1.0, -1.0, 2.0])
    _, fail = oracle.chol(A)
    assert fail == 3
    _, fail = oracle.chol(A, 2.0)  # shift makes it SPD
    assert fail == 0
    A2 = np.eye(3)
    A2[1, 1] = np.nan
    assert oracle.chol(A2)[1] == 2
    # exactly singular: radicand 0 counts as breakdown
    v = np.array([[1.0, 1.0], [1.0, 1.0]])
    assert oracle.chol(v)[1] == 2


def test_trsm_exact_on_integers():
    rng = np.random.default_rng(3)
    for n in (1, 3, 8, 17):
        R = _int_upper(n, rng)
        Qi = rng.integers(-20, 21, size=(41, n)).astype(np.float64)
        X = Qi @ R
        assert np.array_equal(oracle.trsm(X, R), Qi)


def test_trmm_exact_on_integers():
    rng = np.random.default_rng(4)
    n = 9
    A = np.triu(rng.integers(-5, 6, size=(n, n))).astype(np.float64)
    B = np.triu(rng.integers(-5, 6, size=(n, n))).astype(np.float64)
    assert np.array_equal(oracle.trmm(A, B), (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64))


# --------------------------------------------------------------------------- shift, pinned by printed values

@pytest.mark.parametrize("key", ["table1", "table2"])
def test_pass1_condition_matches_printed_table(golden, key):
    """kappa_2(Q^(1)) printed in Tables 1-2 pins Eq. (finds2): both the mn and
    the n(n+1) terms and the factor 11 (Table 2 has m = n, so dropping n(n+1)
    would be off by 30%)."""
    g = golden[key]
    m, n, kappa = g["m"], g["n"], g["kappa"]
    X = testmat(m, n, kappa, seed=11)
    s = oracle.shift(m, n, 1.0)  # ||X||_2 = 1 by construction
    R1, fail = oracle.chol(oracle.gram(X), s)
    assert fail == 0
    k1 = np.linalg.cond(oracle.trsm(X, R1))
    assert abs(k1 / g["kappa_Q"][0] - 1.0) < 0.01


def test_shift_remark_value(golden):
    """The remark's ~6.1e-11 (m=1000, n=50) is 11 mn u; the formula with
    n(n+1) gives 6.42e-11. The 5% gap is the paper's rounding of its own
    example; we follow the formula (Eq. finds2), which Tables 1-2 confirm."""
    g = golden["shift_remark"]
    s = oracle.shift(g["m"], g["n"], 1.0)
    assert 1.0 < s / g["s_printed"] < 1.07


def test_oblique_shift_matches_table3(golden):
    """Table 3's sqrt(alpha kappa_2(B)) = 8.41e-2 pins Eq. (finds2B)."""
    g = golden["table3"]
    alpha = oracle.shift_oblique(g["m"], g["n"], 1.0, 1.0)
    assert abs(np.sqrt(alpha * g["kappa_b"]) / g["sqrt_alpha_kappa_b"] - 1.0) < 0.005
    # scaling: s is linear in ||X||^2 and in ||B||
    assert oracle.shift_oblique(300, 30, 3.0, 5.0) == pytest.approx(15.0 * alpha, rel=1e-15)
    assert oracle.shift(77, 5, 2.5) == pytest.approx(2.5 * oracle.shift(77, 5, 1.0), rel=1e-15)


# --------------------------------------------------------------------------- per-pass behaviour (Tables 1-3)

@pytest.mark.parametrize("key", ["table1", "table2"])
def test_per_pass_magnitudes_tables_1_2(golden, key):
    g = golden[key]
    m, n, kappa = g["m"], g["n"], g["kappa"]
    X = testmat(m, n, kappa, seed=12)
    Q, R, st, tr = oracle.scqr3(X, normx2=1.0)
    assert st == 0 and tr["passes"] == 3 and tr["shifted"] == [1, 0, 0]
    # replay the three passes with the building blocks to look at each iterate
    Qk = X.copy()
    for p in range(3):
        Rt, fail = oracle.chol(oracle.gram(Qk), tr["s"][p])
        assert fail == 0
        Qk = oracle.trsm(Qk, Rt)
        o = orth2(Qk)
        want = g["orth2"][p]
        if p == 0:
            assert 0.9 < o < 1.0 + 1e-6  # ||Q^T Q - I||_2 = 1 - lambda_min
        elif p == 1:
            assert want / 30 < o < want * 30
        else:
            assert o < 10 * want and o < 1e-14
        if p >= 1:
            assert np.linalg.cond(Qk) < 1.2
    assert np.array_equal(Qk, Q)


def test_per_pass_magnitudes_table3(golden):
    g = golden["table3"]
    m, n = g["m"], g["n"]
    X = testmat(m, n, g["kappa_x"], seed=13)
    B = dense_spd(m, g["kappa_b"], seed=14)
    Bblk = B[None]
    sB = np.linalg.svd(B, compute_uv=False)
    Bh = (np.linalg.eigh(B)[1] * np.sqrt(np.linalg.eigvalsh(B))) @ np.linalg.eigh(B)[1].T

    def measure(Qk):
        smin = np.linalg.svd(Bh @ Qk, compute_uv=False).min()
        return np.linalg.norm(Qk, 2) * np.sqrt(sB.max()) / smin

    Q, R, st, tr = oracle.scqr3(X, Bblk, normx2=1.0, normb=float(sB.max()))
    assert st == 0 and tr["passes"] == 3
    Qk = X.copy()
    for p in range(3):
        A, _ = oracle.gram_oblique(Qk, Bblk)
        Rt, fail = oracle.chol(A, tr["s"][p])
        assert fail == 0
        Qk = oracle.trsm(Qk, Rt)
        mk = measure(Qk)
        assert g["measure"][p] / 3 < mk < g["measure"][p] * 3
        ob = np.linalg.norm(Qk.T @ B @ Qk - np.eye(n), 2)
        if p == 1:
            assert g["orth2_b"][1] / 30 < ob < 1.0
        if p == 2:
            assert ob < 10 * g["orth2_b"][2]
    assert resid(X, Q, R) < 16 * n * n * U * np.sqrt(g["kappa_b"]) ** 3


# --------------------------------------------------------------------------- closed forms and invariants

@pytest.mark.parametrize("kappa", [1e6, 1e9, 1e12, 1e14])
def test_pass1_condition_closed_form(kappa):
    """In exact arithmetic R1^T R1 = V(S^2 + sI)V^T, so the singular values of
    X R1^{-1} are sigma_i / sqrt(sigma_i^2 + s) (Thm. on kappa reduction)."""
    m, n = 500, 12
    Uf, sig, V = testmat_factors(m, n, kappa, seed=21)
    X = (Uf * sig) @ V.T
    s = oracle.shift(m, n, 1.0)
    R1, fail = oracle.chol(oracle.gram(X), s)
    assert fail == 0
    sv = sig / np.sqrt(sig ** 2 + s)
    want = sv.max() / sv.min()
    got = np.linalg.cond(oracle.trsm(X, R1))
    assert abs(got / want - 1.0) < 0.05
    # bound of Thm. (eq:kap2): kappa(Q1) <= 2 sqrt(3) sqrt(1 + alpha kappa^2)
    assert got <= 2 * np.sqrt(3) * np.sqrt(1 + s * kappa ** 2)


@pytest.mark.parametrize("m,n", [(300, 10), (1000, 30), (64, 64), (2000, 7)])
@pytest.mark.parametrize("kappa", [1e2, 1e8, 1e12, 1e15])
def test_end_to_end_bounds(m, n, kappa):
    """Thm. (maincholqr3): ||Q^T Q - I||_F <= 6{mn + n(n+1)}u and
    ||QR - X||_F / ||X||_2 <= 15 n^2 u; R upper triangular, diag(R) > 0."""
    X = testmat(m, n, kappa, seed=int(np.log10(kappa)) * 7 + n)
    Q, R, st, tr = oracle.scqr3(X)
    assert st == 0
    assert np.array_equal(np.tril(R, -1), np.zeros((n, n)))
    assert (np.diag(R) > 0).all()
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 6 * (m * n + n * (n + 1)) * U
    assert np.linalg.norm(Q @ R - X) / np.linalg.norm(X, 2) <= 15 * n * n * U
    assert tr["shifted"][0] == 1 and tr["shifted"][-2:] == [0, 0]


@pytest.mark.parametrize("kappa", [1e1, 1e4, 1e8])
@pytest.mark.parametrize("m,n", [(50, 50), (200, 13), (300, 32)])
def test_matches_householder_qr(m, n, kappa):
    """Brute force: the QR factorization with diag(R) > 0 is unique; LAPACK's
    Householder QR gives it to within kappa*u."""
    X = testmat(m, n, kappa, seed=31 + n)
    Q, R, st, _ = oracle.scqr3(X)
    assert st == 0
    Qh, Rh = signfix_qr(X)
    tol = 50 * n * kappa * U
    assert np.linalg.norm(R - Rh) / np.linalg.norm(Rh) < tol
    assert np.linalg.norm(Q - Qh) < tol * np.sqrt(n)


@pytest.mark.parametrize("kappa", [1e2, 1e6, 1e8])
def test_R_equals_R_factor_of_sigma_vt(kappa):
    """X = U S V^T with orthonormal U gives R = R-factor of S V^T exactly."""
    m, n = 3000, 24
    Uf, sig, V = testmat_factors(m, n, kappa, seed=41)
    X = (Uf * sig) @ V.T
    _, R, st, _ = oracle.scqr3(X)
    assert st == 0
    _, Rx = signfix_qr(sig[:, None] * V.T)
    assert np.linalg.norm(R - Rx) / np.linalg.norm(Rx) < 100 * n * kappa * U


def test_accumulation_order_R_is_Rtilde_times_R():
    """R := Rt R (the update of Alg. 2): the reversed product would break X = QR."""
    X = testmat(400, 9, 1e11, seed=5)
    Q, R, st, tr = oracle.scqr3(X)
    assert st == 0 and tr["passes"] >= 3
    assert resid(X, Q, R) < 1e-15 * 9


def test_q_may_alias_x_and_trace_values():
    X = testmat(256, 16, 1e10, seed=6)
    Q, R, st, tr = oracle.scqr3(X.copy())
    assert tr["s"][0] == pytest.approx(oracle.shift(256, 16, np.trace(X.T @ X)), rel=1e-12)
    assert tr["s"][1:] == [0.0] * (tr["passes"] - 1)


# --------------------------------------------------------------------------- Alg. 2 breakdown rule

def test_extra_shifted_pass_when_cholqr_breaks_down():
    """kappa = 1e15 at m=20000, n=32: kappa(Q1) ~ sqrt(alpha) kappa ~ 1e11 >
    u^{-1/2}, so the plain Cholesky of pass 2 breaks down and Alg. 2 shifts
    again; two plain passes then finish."""
    m, n = 20000, 32
    X = testmat(m, n, 1e15, seed=7)
    Q, R, st, tr = oracle.scqr3(X)
    assert st == 0
    assert tr["passes"] == 4 and tr["shifted"] == [1, 1, 0, 0]
    assert tr["unshifted_fail"][1] > 0
    # recursive summation over 20000 rows: about sqrt(m) u in practice
    assert orth2(Q) < 1e-13 and resid(X, Q, R) < 1e-15


def test_repeated_small_singular_values():
    m, n = 5000, 32
    X = testmat(m, n, 0.0, seed=8, sigma=repeated_small_sigma(n, 8, 1e-14, 1e7))
    Q, R, st, tr = oracle.scqr3(X)
    assert st == 0 and tr["shifted"][0] == 1
    assert orth2(Q) < 1e-13 and resid(X, Q, R) < 1e-15


def test_max_passes_reported():
    m, n = 20000, 32
    X = testmat(m, n, 1e15, seed=7)
    _, _, st, tr = oracle.scqr3(X, max_passes=3)
    assert st == oracle.E_MAXPASS and tr["passes"] == 3


def test_argument_and_input_errors():
    X = np.ones((4, 5))
    assert oracle.scqr3(X)[2] == oracle.E_ARG  # m < n
    X = testmat(50, 4, 10.0, seed=9)
    X[3, 2] = np.nan
    assert oracle.scqr3(X)[2] == oracle.E_NONFINITE
    Z = testmat(50, 4, 10.0, seed=9)
    Z[:, 2] = 0.0  # rank deficient: even the shifted pass leaves the column zero
    st = oracle.scqr3(Z)[2]
    assert st != 0


# --------------------------------------------------------------------------- oblique reductions

def test_oblique_diagonal_B_reduces_to_standard():
    """B = D diagonal: Q_B = D^{-1/2} Qt, R_B = Rt with Qt Rt = QR(D^{1/2} X)."""
    m, n = 400, 10
    rng = np.random.default_rng(51)
    d = rng.uniform(0.5, 4.0, size=m)
    X = testmat(m, n, 1e6, seed=52)
    Q, R, st, _ = oracle.scqr3(X, d.reshape(m, 1, 1))
    assert st == 0
    Qt, Rt = signfix_qr(np.sqrt(d)[:, None] * X)
    assert np.linalg.norm(R - Rt) / np.linalg.norm(Rt) < 1e-9
    assert np.linalg.norm(Q - Qt / np.sqrt(d)[:, None]) < 1e-9
    assert np.linalg.norm(Q.T @ (d[:, None] * Q) - np.eye(n), 2) < 1e-14


def test_oblique_block_diagonal_reduces_to_standard():
    """B = L L^T blockwise: Q_B = L^{-T} Qt, R_B = Rt with Qt Rt = QR(L^T X)."""
    m, n, bs = 512, 16, 8
    Bblk = block_diag_spd(m, bs, seed=53)
    X = testmat(m, n, 1e6, seed=54)
    Q, R, st, tr = oracle.scqr3(X, Bblk)
    assert st == 0
    L = np.linalg.cholesky(Bblk)  # lower, per block
    LtX = np.einsum("kji,kjn->kin", L, X.reshape(-1, bs, n)).reshape(m, n)
    Qt, Rt = signfix_qr(LtX)
    assert np.linalg.norm(R - Rt) / np.linalg.norm(Rt) < 1e-8
    QB = np.linalg.solve(np.transpose(L, (0, 2, 1)), Qt.reshape(-1, bs, n)).reshape(m, n)
    assert np.linalg.norm(Q - QB) / np.linalg.norm(QB) < 1e-8
    BQ = np.einsum("kij,kjn->kin", Bblk, Q.reshape(-1, bs, n)).reshape(m, n)
    assert np.linalg.norm(Q.T @ BQ - np.eye(n), 2) < 1e-13
    # the shift used ||B||_2 bounded by the largest block Frobenius norm
    assert tr["s"][0] == pytest.approx(
        oracle.shift_oblique(m, n, float((X * X).sum()), oracle.normb_bound(Bblk)), rel=1e-12)


def test_normb_bound_is_an_upper_bound():
    Bblk = block_diag_spd(64, 8, seed=55)
    lam = max(np.linalg.eigvalsh(b).max() for b in Bblk)
    nb = oracle.normb_bound(Bblk)
    assert lam <= nb <= np.sqrt(8) * lam


def test_deterministic():
    X = testmat(1000, 20, 1e12, seed=56)
    a = oracle.scqr3(X)
    b = oracle.scqr3(X)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_geometric_sigma():
    s = geometric_sigma(5, 1e4)
    assert s[0] == 1.0 and s[-1] == pytest.approx(1e-4)
    assert np.allclose(s[1:] / s[:-1], 10 ** -1.0)


# --------------------------------------------------------------------------- options: the smaller shift of the
# remark in Sec. 6.1 and the adaptive Alg. 2

def _fig3_input(seed):
    """The setup of the Sec. 6.1 remark (its Fig. 3): m=1000, n=50, kappa 1e15, ||X||_2=1."""
    Uf, sig, V = testmat_factors(1000, 50, 1e15, seed=seed)
    return (Uf * sig) @ V.T, sig


def test_small_shift_reduces_passes_fig3_setup():
    """With the safe shift 11{mn+n(n+1)}u the remark notes that kappa(Q^(1)) is
    too large for CholeskyQR2 and more passes follow (here one more shifted
    pass). With s = c u ||X||^2 (c = 100) the first Cholesky succeeds, s is
    exactly c u, kappa(Q^(1)) follows sigma_i / sqrt(sigma_i^2 + s) from the SVD
    of X, and CholeskyQR2 finishes: three passes in all."""
    X, sig = _fig3_input(3)
    m, n = X.shape
    _, _, st, tr = oracle.scqr3(X, normx2=1.0)
    assert st == 0 and tr["passes"] == 4 and tr["shifted"] == [1, 1, 0, 0]
    Q, R, st, tr = oracle.scqr3(X, normx2=1.0, shift_scale=100.0)
    assert st == 0 and tr["passes"] == 3 and tr["shifted"] == [1, 0, 0]
    assert tr["s"][0] == 100.0 * U
    R1, fail = oracle.chol(oracle.gram(X), tr["s"][0])
    assert fail == 0
    sv = sig / np.sqrt(sig ** 2 + tr["s"][0])
    assert abs(np.linalg.cond(oracle.trsm(X, R1)) / (sv.max() / sv.min()) - 1.0) < 0.05
    assert orth2(Q) < 1e-14 and resid(X, Q, R) < 1e-15


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_small_shift_falls_back_when_shifted_gram_is_indefinite(seed):
    """The remark gives no guarantee for chol(A + u||X||^2 I). On the Fig. 3
    setup the computed Gram matrix has an eigenvalue near -2u (its rounding
    error), so A + uI is indefinite (numpy's eigvalsh, independent of the
    oracle), the Cholesky must break down, and the safe shift of Eq. (finds2)
    is used instead, exactly."""
    X, _ = _fig3_input(seed)
    m, n = X.shape
    A = oracle.gram(X)
    assert np.linalg.eigvalsh(A + U * np.eye(n)).min() < 0.0
    _, _, st, tr = oracle.scqr3(X, normx2=1.0, shift_scale=1.0)
    assert st == 0
    assert tr["s"][0] == oracle.shift(m, n, 1.0)


def test_small_shift_oblique_scales_with_normb():
    """The oblique form of the smaller shift is c u ||X||^2 ||B||."""
    m, n, bs = 512, 16, 8
    Bblk = block_diag_spd(m, bs, seed=57)
    X = testmat(m, n, 1e6, seed=58)
    _, _, st, tr = oracle.scqr3(X, Bblk, normx2=2.0, normb=3.0, shift_scale=1e4)
    assert st == 0 and tr["s"][0] == 1e4 * U * 2.0 * 3.0


@pytest.mark.parametrize("key", ["table1", "table2"])
def test_alg2_reproduces_table_iterates(golden, key):
    """Tables 1-2 list three iterates of Alg. 2: the plain Cholesky of X^T X
    breaks down (kappa^2 >> 1/u), the shifted pass follows, then two plain
    passes, after which ||Q^T Q - I||_F is at rounding level and the loop ends.
    The computation is then pass for pass the one of Alg. 3, bit for bit."""
    g = golden[key]
    X = testmat(g["m"], g["n"], g["kappa"], seed=12)
    Q2, R2, st2, tr2 = oracle.scqr3(X, normx2=1.0, algorithm=2)
    assert st2 == 0 and tr2["passes"] == 3 and tr2["shifted"] == [1, 0, 0]
    assert tr2["unshifted_fail"][0] > 0
    Q3, R3, st3, tr3 = oracle.scqr3(X, normx2=1.0)
    assert np.array_equal(Q2, Q3) and np.array_equal(R2, R3) and tr2["s"] == tr3["s"]


@pytest.mark.parametrize("kappa,passes", [(1.0, 1), (1e3, 2), (1e7, 2)])
def test_alg2_stops_when_orthogonal_enough(kappa, passes):
    """Alg. 2 needs no shift for kappa(X) < u^{-1/2}: one plain CholeskyQR when
    X is already orthonormal, two (CholeskyQR2) otherwise. The stopping test
    is replayed with the building blocks: the iterate it stops at is the first
    whose ||Q^T Q - I||_F is below 6{mn+n(n+1)}u, and the one before is not."""
    m, n = 2000, 20
    X = testmat(m, n, kappa, seed=1)
    Q, R, st, tr = oracle.scqr3(X, algorithm=2)
    assert st == 0 and tr["passes"] == passes and tr["shifted"] == [0] * passes
    tol = 6 * (m * n + n * (n + 1)) * U
    Qk = X.copy()
    devs = []
    for p in range(passes):
        Rt, fail = oracle.chol(oracle.gram(Qk), 0.0)
        assert fail == 0
        Qk = oracle.trsm(Qk, Rt)
        devs.append(np.linalg.norm(oracle.gram(Qk) - np.eye(n)))
    assert np.array_equal(Qk, Q)
    assert devs[-1] <= tol and all(d > tol for d in devs[:-1])
    assert resid(X, Q, R) < 1e-15


def test_alg2_printed_tolerance_is_below_gram_rounding():
    """With the printed tolerance sqrt(n) u the test is compared with the
    computed Gram matrix, whose own rounding error (about sqrt(m) u per entry)
    is larger, so the iteration runs to the pass limit."""
    m, n = 1000, 30
    X = testmat(m, n, 1e12, seed=12)
    Q, _, st, tr = oracle.scqr3(X, normx2=1.0, algorithm=2, tol=np.sqrt(n) * U, max_passes=5)
    assert st == oracle.E_MAXPASS and tr["passes"] == 5
    assert np.linalg.norm(oracle.gram(Q) - np.eye(n)) > np.sqrt(n) * U
    assert orth2(Q) < 1e-14


def test_option_arguments_checked():
    X = testmat(100, 4, 10.0, seed=9)
    assert oracle.scqr3(X, algorithm=1)[2] == oracle.E_ARG
    assert oracle.scqr3(X, algorithm=4)[2] == oracle.E_ARG


@pytest.mark.parametrize("m,n", [(1000, 30), (20000, 64)])
@pytest.mark.parametrize("kappa", [1e16, 1e18, 1e20])
def test_alg2_beyond_one_over_u(m, n, kappa):
    """Sec. 4 observes that Alg. 2 may work even for kappa(X) > 1/u (no
    guarantee): shifted passes repeat until kappa(Q) allows CholeskyQR2. The
    orthogonality and residual bounds of Thm. (maincholqr3) still hold, every
    shifted pass precedes every plain one, and two plain passes end it."""
    X = testmat(m, n, kappa, seed=77)
    Q, R, st, tr = oracle.scqr3(X, normx2=1.0, algorithm=2, max_passes=8)
    assert st == 0
    k = tr["passes"]
    assert k >= 4 and tr["shifted"] == [1] * (k - 2) + [0, 0]
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 6 * (m * n + n * (n + 1)) * U
    assert np.linalg.norm(Q @ R - X) / np.linalg.norm(X, 2) <= 15 * n * n * U


# --------------------------------------------------------------------------- sparse B in CSR form (Sec. 7.2)

def _dense_to_csr(B):
    m = B.shape[0]
    rows, cols = np.nonzero(B)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr), cols.astype(np.int32), B[rows, cols].astype(np.float64)


def test_gram_csr_exact_on_integers():
    """A = X^T (B X) on small integers is exact in FP64: compare with int64."""
    rng = np.random.default_rng(61)
    m, n = 40, 7
    Bi = rng.integers(-3, 4, size=(m, m)) * (rng.random((m, m)) < 0.15)
    Bi = Bi + Bi.T + np.diag(rng.integers(1, 9, size=m))
    Xi = rng.integers(-4, 5, size=(m, n))
    A, f = oracle.gram_csr(Xi.astype(float), _dense_to_csr(Bi.astype(float)))
    want = Xi.T @ (Bi @ Xi)
    assert np.array_equal(np.triu(A), np.triu(want).astype(float))
    assert np.array_equal(A, A.T)
    assert f == float((Xi * Xi).sum())


def test_normb_csr_is_max_abs_row_sum_and_bounds_norm():
    from paper_1809_11085_gb300.testmat import csr_to_dense, random_spd_csr

    csr = random_spd_csr(500, 3, 1e3, seed=62)
    B = csr_to_dense(csr, 500)
    nb = oracle.normb_csr(csr)
    assert nb == pytest.approx(np.abs(B).sum(axis=1).max(), rel=1e-14)
    assert np.linalg.eigvalsh(B).max() <= nb


def test_csr_block_diagonal_matches_block_path():
    """A block-diagonal B stored as CSR (same entry order) is the same
    arithmetic as the block-diagonal form: bitwise equal results."""
    m, n, bs = 256, 12, 8
    Bblk = block_diag_spd(m, bs, seed=63)
    B = np.zeros((m, m))
    for k in range(m // bs):
        B[k * bs:(k + 1) * bs, k * bs:(k + 1) * bs] = Bblk[k]
    X = testmat(m, n, 1e8, seed=64)
    nb = 3.7
    Q1, R1, st1, tr1 = oracle.scqr3(X, Bblk, normb=nb)
    Q2, R2, st2, tr2 = oracle.scqr3(X, normb=nb, csr=_dense_to_csr(B))
    assert st1 == st2 == 0
    assert np.array_equal(Q1, Q2) and np.array_equal(R1, R2) and tr1 == tr2


@pytest.mark.parametrize("dims,kappa_b", [((18, 20), 1e3), ((6, 7, 8), 1e2)])
def test_csr_laplacian_reduces_to_standard(dims, kappa_b):
    """B = L L^T (dense Cholesky of the sparse Laplacian, numpy): Q_B = L^{-T} Qt
    and R_B = Rt with Qt Rt = QR(L^T X); the shift is Eq. (finds2B) with the
    max absolute row sum for ||B||_2."""
    from paper_1809_11085_gb300.testmat import csr_to_dense, laplacian_csr

    csr = laplacian_csr(dims, kappa_b)
    m = int(np.prod(dims))
    n = 10
    B = csr_to_dense(csr, m)
    X = testmat(m, n, 1e6, seed=65)
    Q, R, st, tr = oracle.scqr3(X, csr=csr)
    assert st == 0
    L = np.linalg.cholesky(B)
    Qt, Rt = signfix_qr(L.T @ X)
    assert np.linalg.norm(R - Rt) / np.linalg.norm(Rt) < 1e-8
    QB = np.linalg.solve(L.T, Qt)
    assert np.linalg.norm(Q - QB) / np.linalg.norm(QB) < 1e-8
    assert np.linalg.norm(Q.T @ B @ Q - np.eye(n), 2) < 1e-13
    assert tr["s"][0] == pytest.approx(
        oracle.shift_oblique(m, n, float((X * X).sum()), float(np.abs(B).sum(axis=1).max())), rel=1e-12)


def test_csr_random_pattern_bounds():
    """Thm. (Bsta): ||Q^T B Q - I||_F <= 8[m sqrt(mn) u + n(n+1) u] kappa(B) and
    ||QR - X||_F / ||X||_2 <= 16 n^2 u kappa(B)^{3/2} (here ||X||_2 = 1; the
    theorem's condition 80 kappa(B)(m sqrt(mn) u + n(n+1) u) <= 1 holds)."""
    from paper_1809_11085_gb300.testmat import csr_to_dense, random_spd_csr

    m, n = 2000, 16
    csr = random_spd_csr(m, 3, 1e3, seed=66)
    B = csr_to_dense(csr, m)
    ev = np.linalg.eigvalsh(B)
    kb = ev.max() / ev.min()
    X = testmat(m, n, 1e10, seed=67)
    Q, R, st, tr = oracle.scqr3(X, normx2=1.0, csr=csr)
    assert st == 0 and tr["shifted"][0] == 1
    assert np.linalg.norm(Q.T @ B @ Q - np.eye(n)) <= 8 * (m * np.sqrt(m * n) * U + n * (n + 1) * U) * kb
    assert 80 * kb * (m * np.sqrt(m * n) * U + n * (n + 1) * U) <= 1
    assert np.linalg.norm(Q @ R - X) <= 16 * n * n * U * kb ** 1.5


# ------------------------------------------------------------------ the 2-norm estimate of the shift

def test_normest2_matches_eigvalsh():
    """The power method's Rayleigh quotient converges to lambda_max (here with
    a spectral gap of at least 10%: to within 1e-10 of numpy's eigvalsh)."""
    rng = np.random.default_rng(31)
    for n in (1, 2, 7, 32, 64):
        Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = np.sort(rng.uniform(0.0, 0.9, size=n))
        lam[-1] = 1.0 + rng.uniform(0.0, 5.0)
        A = (Qm * lam) @ Qm.T
        A = (A + A.T) / 2
        est = oracle.normest2(A)
        assert abs(est - np.linalg.eigvalsh(A).max()) <= 1e-10 * lam[-1]


def test_two_norm_estimate_recovers_table1_shift():
    """With ||X||_2 = 1 (the testmat construction), the estimated ||X||_2^2 is
    1 to rounding, so the first shift is Eq. (finds2) with ||X||_2 = 1, as when
    the caller passes norm_x2 = 1, and kappa(Q_1) of Table 1 follows."""
    m, n, kappa = 1000, 30, 1e12
    X = testmat(m, n, kappa, seed=1551)
    _, _, st1, tr1 = oracle.scqr3(X, normx2=1.0)
    Q, R, st, tr = oracle.scqr3(X, normx2=oracle.TWO_NORM_EST)
    assert st == 0 and st1 == 0
    assert abs(tr["norm2"][0] - 1.0) <= 1e-12
    assert abs(tr["s"][0] - oracle.shift(m, n, 1.0)) <= 1e-12 * tr["s"][0]
    assert tr["passes"] == tr1["passes"]
    # every later shifted pass uses its own iterate's estimate; results keep the bounds
    assert np.linalg.norm(Q.T @ Q - np.eye(n), 2) <= 6 * (m * n + n * (n + 1)) * 2.0 ** -53
