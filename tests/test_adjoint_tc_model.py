"""Exact-arithmetic model (numpy, CPU) of the tensor-core adjoint's data flow.

The tensor-core adjoint holds the iterate of reverse pass k as
Z = [Q_k | Qbar_k J] (J reverses the column order) and runs three identities:
  * t J = Qbar_k J - Q_k Bt with Bt = -2 P_k J          (t = Qbar_k + 2 Q_k P_k)
  * (Qbar_{k-1} J) U = t J with U = J R_k^T J, U(a, b) = R_k(n-1-b, n-1-a),
    upper triangular                                    (Qbar_{k-1} R_k^T = t)
  * M_{k-1}(r, j) = G(r, 2n-1-j) with G = Z^T Z of the new Z
                                                         (M_{k-1} = Q_{k-1}^T Qbar_{k-1})
This model runs those steps with numpy primitives in the kernels' index
conventions and compares the result with the pass-wise oracle adjoint: a
wrong reversal, a transposed U or a misplaced block of G fails it.
"""
import numpy as np
import pytest
import scipy.linalg as sl

from oracle.adjoint import passwise_adjoint, phi
from paper_1809_11085_gb300.testmat import testmat


def model_adjoint(Q, Rks, dQ, dR):
    n = Q.shape[1]
    eye = np.eye(n)

    def prod(ms):
        o = eye.copy()
        for A in ms:
            o = A @ o
        return o

    Z = np.hstack([Q, dQ[:, ::-1]])
    G = Z.T @ Z
    for k in range(len(Rks), 0, -1):
        Rk = Rks[k - 1]
        M = np.array([[G[r, 2 * n - 1 - j] for j in range(n)] for r in range(n)])
        L, Ra = prod(Rks[k:]), prod(Rks[: k - 1])
        Rb = np.triu(L.T @ dR @ Ra.T - np.linalg.solve(Rk, M.T).T)
        Pk = phi(Rb @ Rk.T)
        Pk = 0.5 * (Pk + Pk.T)
        Bt = np.array([[-2.0 * Pk[a, n - 1 - b] for b in range(n)] for a in range(n)])
        Bq = -np.triu(Rk)
        U = np.zeros((n, n))
        for a in range(n):
            for b in range(a, n):
                U[a, b] = Rk[n - 1 - b, n - 1 - a]
        t_rev = Z[:, n:] - Z[:, :n] @ Bt
        y_rev = sl.solve_triangular(U, t_rev.T, trans="T", lower=False).T  # y_rev U = t_rev
        Z = np.hstack([-(Z[:, :n] @ Bq), y_rev])
        G = Z.T @ Z
    return Z[:, n:][:, ::-1]


@pytest.mark.parametrize("n", [1, 3, 20, 64])
def test_reversed_layout_matches_passwise_adjoint(n):
    m = 400
    rng = np.random.default_rng(40 + n)
    X = testmat(m, n, 1e4, seed=41 + n)
    Q, R = np.linalg.qr(X)
    s = np.sign(np.diag(R))
    Q, R = Q * s, (R.T * s).T
    R2 = np.triu(rng.standard_normal((n, n))) * 0.01 + np.eye(n)
    R3 = np.triu(rng.standard_normal((n, n))) * 0.01 + np.eye(n)
    Rks = [np.linalg.solve(R3 @ R2, R), R2, R3]  # R3 R2 R1 = R, each upper triangular
    dQ = rng.standard_normal((m, n))
    dR = rng.standard_normal((n, n))
    a = model_adjoint(Q, Rks, dQ, dR)
    b = passwise_adjoint(Q, Rks, dQ, dR)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12
