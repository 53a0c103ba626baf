"""Pins of the gradient references: both adjoints against central finite
differences of the CPU oracle's forward map, and against each other."""
import numpy as np
import pytest

import oracle
from oracle.adjoint import passwise_adjoint, qr_adjoint, qr_adjoint_rows
from paper_1809_11085_gb300.testmat import testmat


def replay_passes(X, tr):
    """Per-pass factors R_1..R_P of the oracle's factorization of X."""
    Qk = X.copy()
    Rks = []
    for p in range(tr["passes"]):
        Rt, fail = oracle.chol(oracle.gram(Qk), tr["s"][p])
        assert fail == 0
        Qk = oracle.trsm(Qk, Rt)
        Rks.append(Rt)
    return Qk, Rks


def loss(X, W1, W2):
    Q, R, st, _ = oracle.scqr3(X)
    assert st == 0
    return float(np.sum(W1 * Q) + np.sum(W2 * R))


@pytest.mark.parametrize("m,n,kappa", [(8, 3, 5.0), (30, 5, 1e2), (60, 7, 1e3)])
def test_closed_form_matches_central_differences(m, n, kappa):
    rng = np.random.default_rng(100 + n)
    X = testmat(m, n, kappa, seed=200 + n)
    W1 = rng.standard_normal((m, n))
    W2 = rng.standard_normal((n, n))
    Q, R, st, _ = oracle.scqr3(X)
    G = qr_adjoint(Q, R, W1, W2)
    h = 1e-6
    for _ in range(4):
        D = rng.standard_normal((m, n))
        fd = (loss(X + h * D, W1, W2) - loss(X - h * D, W1, W2)) / (2 * h)
        an = float(np.sum(G * D))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) * kappa, (fd, an)


def test_full_gradient_by_finite_differences_tiny():
    m, n = 6, 3
    rng = np.random.default_rng(7)
    X = testmat(m, n, 3.0, seed=8)
    W1 = rng.standard_normal((m, n))
    W2 = np.triu(rng.standard_normal((n, n)))
    Q, R, st, _ = oracle.scqr3(X)
    G = qr_adjoint(Q, R, W1, W2)
    h = 1e-6
    F = np.zeros_like(X)
    for i in range(m):
        for j in range(n):
            E = np.zeros_like(X)
            E[i, j] = h
            F[i, j] = (loss(X + E, W1, W2) - loss(X - E, W1, W2)) / (2 * h)
    assert np.max(np.abs(F - G)) < 1e-7 * np.max(np.abs(G))


@pytest.mark.parametrize("kappa", [1e2, 1e5, 1e8, 1e12])
def test_passwise_equals_closed_form(kappa):
    m, n = 400, 12
    rng = np.random.default_rng(9)
    X = testmat(m, n, kappa, seed=10)
    Q, R, st, tr = oracle.scqr3(X)
    assert st == 0
    Qr, Rks = replay_passes(X, tr)
    assert np.array_equal(Qr, Q)
    dQ = rng.standard_normal((m, n))
    dR = rng.standard_normal((n, n))
    a = qr_adjoint(Q, R, dQ, dR)
    b = passwise_adjoint(Q, Rks, dQ, dR)
    rel = np.linalg.norm(a - b) / np.linalg.norm(a)
    assert rel < 1e3 * kappa * 2.0 ** -53, rel


def test_shift_is_irrelevant_to_the_map():
    """Same X, different pass-1 shifts: same (Q, R) up to rounding, so the
    shift carries no gradient (it is held fixed in the adjoint)."""
    X = testmat(300, 8, 1e6, seed=11)
    Q1, R1, _, _ = oracle.scqr3(X)
    Q2, R2, _, _ = oracle.scqr3(X, normx2=37.0)  # a much larger shift
    assert np.linalg.norm(R1 - R2) / np.linalg.norm(R1) < 1e-9
    assert np.linalg.norm(Q1 - Q2) < 1e-9


def test_row_sampled_closed_form_equals_full():
    """qr_adjoint_rows (M summed over row chunks, selected rows) gives the
    selected rows of qr_adjoint, for uneven chunks and with or without dR."""
    rng = np.random.default_rng(77)
    m, n = 1000, 12
    X = rng.standard_normal((m, n)) @ np.diag(np.logspace(0, -4, n))
    Q, R = np.linalg.qr(X)
    s = np.sign(np.diag(R))
    Q, R = Q * s, (R.T * s).T
    dQ = rng.standard_normal((m, n))
    rows = np.array([0, 1, 17, 499, 998, 999])
    for dR in (rng.standard_normal((n, n)), None):
        full = qr_adjoint(Q, R, dQ, dR)
        bounds = [0, 1, 300, 301, 777, m]
        chunks = ((Q[a:b], dQ[a:b]) for a, b in zip(bounds[:-1], bounds[1:]))
        got = qr_adjoint_rows(R, dR, chunks, Q[rows], dQ[rows])
        assert np.allclose(got, full[rows], rtol=1e-12, atol=1e-12 * np.abs(full).max())
