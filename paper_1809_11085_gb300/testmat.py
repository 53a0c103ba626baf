"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

Holds none of the factorization's arithmetic: it only draws matrices.

* ``testmat``: X = U diag(sigma) V^T (Sec. 6.1, the randsvd-like construction
  of the numerical experiments), with U the orthonormal factor of a seeded
  Gaussian m x n matrix, V a Haar-distributed n x n orthogonal matrix (sign-
  fixed QR of a Gaussian, Mezzadri 2007) and sigma geometric from 1 down to
  1/kappa, so ||X||_2 = 1 and kappa_2(X) = kappa.
* ``block_diag_spd``: B = blockdiag(G_j^T G_j + shift I) with seeded Gaussian
  G_j, the block-diagonal SPD inner product used for the oblique variant.
* ``batched_shapes``: the uneven (m_i, n_i, kappa_i) mix of the batched form.

numpy versions serve sizes the CPU oracle can handle; the torch versions draw
the same distributions on a CUDA device for the large cases.
"""
from __future__ import annotations

import numpy as np


def geometric_sigma(n: int, kappa: float) -> np.ndarray:
    """diag(1, s^(1/(n-1)), ..., s) with s = 1/kappa (Sec. 6.1)."""
    if n == 1:
        return np.ones(1)
    return np.power(1.0 / kappa, np.arange(n) / (n - 1.0))


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    G = rng.standard_normal((n, n))
    Qm, Rm = np.linalg.qr(G)
    d = np.sign(np.diag(Rm))
    d[d == 0] = 1.0
    return Qm * d


def testmat(m: int, n: int, kappa: float, seed: int, sigma: np.ndarray | None = None) -> np.ndarray:
    """X = U diag(sigma) V^T, row-major float64, ||X||_2 = max(sigma)."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V = haar_orthogonal(n, rng)
    s = geometric_sigma(n, kappa) if sigma is None else np.asarray(sigma, dtype=np.float64)
    return np.ascontiguousarray((U * s) @ V.T)


def testmat_factors(m: int, n: int, kappa: float, seed: int, sigma: np.ndarray | None = None):
    """(U, sigma, V) of ``testmat`` with the same seed."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V = haar_orthogonal(n, rng)
    s = geometric_sigma(n, kappa) if sigma is None else np.asarray(sigma, dtype=np.float64)
    return U, s, V


def repeated_small_sigma(n: int, n_small: int = 8, small: float = 1e-14, top_kappa: float = 1e7):
    """sigma with the last n_small values equal to `small` and the rest geometric 1 -> 1/top_kappa."""
    s = np.empty(n)
    s[: n - n_small] = geometric_sigma(n - n_small, top_kappa)
    s[n - n_small:] = small
    return s


def block_diag_spd(m: int, bs: int, seed: int, shift: float = 0.1) -> np.ndarray:
    """(m/bs, bs, bs) blocks G^T G + shift*I, G seeded Gaussian."""
    assert m % bs == 0
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m // bs, bs, bs))
    B = np.einsum("kij,kil->kjl", G, G)
    B += shift * np.eye(bs)[None]
    return np.ascontiguousarray(B)


def dense_spd(m: int, kappa: float, seed: int) -> np.ndarray:
    """B = W diag(geometric 1..1/kappa) W^T with W Haar m x m (Sec. 6.1, B = U Sigma U^T)."""
    rng = np.random.default_rng(seed)
    W = haar_orthogonal(m, rng)
    return np.ascontiguousarray((W * geometric_sigma(m, kappa)) @ W.T)


def batched_shapes(count: int, seed: int, m_lo: int = 2000, m_hi: int = 200000,
                   n_choices=(16, 32, 64, 128), logk_lo: float = 2.0, logk_hi: float = 12.0):
    """List of (m_i, n_i, kappa_i) for the batched form."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_lo, m_hi + 1, size=count)
    ns = rng.choice(np.asarray(n_choices), size=count)
    ks = 10.0 ** rng.uniform(logk_lo, logk_hi, size=count)
    return [(int(max(a, b)), int(b), float(c)) for a, b, c in zip(ms, ns, ks)]


# --------------------------------------------------------------------------- torch (device) versions

def testmat_torch(m: int, n: int, kappa: float, seed: int, device="cuda", sigma=None, out=None):
    """Device version of ``testmat`` (same distribution, torch RNG stream).

    U is the Q factor of a seeded Gaussian drawn on the device; the QR is the
    library's Householder QR and is input generation only.
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    G = torch.randn((m, n), generator=g, device=device, dtype=torch.float64)
    U, _ = torch.linalg.qr(G)
    del G
    Gv = torch.randn((n, n), generator=g, device=device, dtype=torch.float64)
    Vq, Vr = torch.linalg.qr(Gv)
    d = torch.sign(torch.diagonal(Vr))
    d[d == 0] = 1.0
    V = Vq * d
    s = torch.as_tensor(geometric_sigma(n, kappa) if sigma is None else np.asarray(sigma),
                        device=device, dtype=torch.float64)
    U.mul_(s)
    if out is None:
        out = torch.empty((m, n), device=device, dtype=torch.float64)
    torch.matmul(U, V.T, out=out)
    del U
    return out, s, V


def block_diag_spd_torch(m: int, bs: int, seed: int, shift: float = 0.1, device="cuda"):
    import torch

    assert m % bs == 0
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    G = torch.randn((m // bs, bs, bs), generator=g, device=device, dtype=torch.float64)
    B = torch.matmul(G.transpose(1, 2), G)
    B += shift * torch.eye(bs, device=device, dtype=torch.float64)
    return B.contiguous()
