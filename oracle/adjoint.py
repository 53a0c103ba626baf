"""Gradient references for shifted CholeskyQR3 (TEST INFRASTRUCTURE ONLY).

Two independent references for dL/dX given dL/dQ and dL/dR:

* ``qr_adjoint``: the closed-form adjoint of the QR map X -> (Q, R) with
  diag(R) > 0 (Walter and Lehmann 2018; Seeger et al. 2017):
      Xbar = (Qbar + Q copyltu(M)) R^{-T},  M = R Rbar^T - Qbar^T Q,
  copyltu(M) = tril(M) + tril(M, -1)^T. In exact arithmetic shifted
  CholeskyQR3 computes this map for any fixed shift (the shift cancels:
  R_2 R_1 is the R factor of X whatever s is), so this is the gradient of
  the factorization itself.
* ``passwise_adjoint``: the chain rule through each CholeskyQR pass in
  reverse (Q_k = Q_{k-1} R_k^{-1}, R_k = chol(Q_{k-1}^T Q_{k-1} + s_k I),
  R = R_P ... R_1), with the shifts held fixed, written with numpy
  primitives step by step:
      Rbar_k  = triu(L_k^T Rbar Racc_{k-1}^T - Q_k^T Qbar_k R_k^{-T})
      P_k     = sym(Phi(Rbar_k R_k^T)),  Phi = upper triangle, diagonal halved
      Qbar_{k-1} = (Qbar_k + 2 Q_k P_k) R_k^{-T},   Q_{k-1} = Q_k R_k
  with L_k = R_P ... R_{k+1} and Racc_{k-1} = R_{k-1} ... R_1.
"""
from __future__ import annotations

import numpy as np


def _solve_right_transpose(B: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Y with Y R^T = B for upper triangular R (i.e. R Y^T = B^T)."""
    return np.linalg.solve(R, B.T).T


def qr_adjoint(Q: np.ndarray, R: np.ndarray, dQ: np.ndarray, dR: np.ndarray | None) -> np.ndarray:
    n = R.shape[0]
    if dR is None:
        dR = np.zeros((n, n))
    M = R @ dR.T - dQ.T @ Q
    C = np.tril(M) + np.tril(M, -1).T
    return _solve_right_transpose(dQ + Q @ C, R)


def qr_adjoint_rows(R: np.ndarray, dR: np.ndarray | None, chunks, Q_rows: np.ndarray,
                    dQ_rows: np.ndarray) -> np.ndarray:
    """Rows of ``qr_adjoint`` for a Q too tall to hold at once: M = R Rbar^T -
    Qbar^T Q is summed over the row chunks (Q_c, Qbar_c) that ``chunks`` yields
    (all rows, each once), then Xbar_i = (Qbar_i + Q_i copyltu(M)) R^{-T} for
    the given rows Q_rows / dQ_rows. The same closed form as qr_adjoint."""
    n = R.shape[0]
    M = R @ (np.zeros((n, n)) if dR is None else dR).T
    for Qc, dQc in chunks:
        M = M - dQc.T @ Qc
    C = np.tril(M) + np.tril(M, -1).T
    return _solve_right_transpose(dQ_rows + Q_rows @ C, R)


def phi(A: np.ndarray) -> np.ndarray:
    """Upper triangle of A with its diagonal halved."""
    return np.triu(A) - 0.5 * np.diag(np.diag(A))


def passwise_adjoint(Q: np.ndarray, Rks: list, dQ: np.ndarray, dR: np.ndarray | None) -> np.ndarray:
    """Chain rule through the passes, from the final Q and the per-pass factors R_1..R_P."""
    P = len(Rks)
    n = Q.shape[1]
    if dR is None:
        dR = np.zeros((n, n))
    eye = np.eye(n)

    def prod(mats):
        out = eye.copy()
        for A in mats:
            out = A @ out
        return out

    Qk = Q.copy()
    Qbar = dQ.copy()
    for k in range(P, 0, -1):
        Rk = Rks[k - 1]
        L = prod(Rks[k:])             # R_P ... R_{k+1}  (applied in order k+1..P)
        Racc = prod(Rks[: k - 1])     # R_{k-1} ... R_1
        Rbar_k = np.triu(L.T @ dR @ Racc.T - _solve_right_transpose(Qk.T @ Qbar, Rk))
        Pk = phi(Rbar_k @ Rk.T)
        Pk = 0.5 * (Pk + Pk.T)
        Qbar = _solve_right_transpose(Qbar + 2.0 * Qk @ Pk, Rk)
        Qk = Qk @ Rk
    return Qbar
