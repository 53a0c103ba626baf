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
* ``laplacian_csr`` / ``random_spd_csr``: sparse SPD B in CSR form for the
  oblique variant with a sparse inner product (Sec. 7.2 uses SuiteSparse
  matrices, which are not available here; these stand in for them): the
  shifted finite-difference Laplacian of a 2-D or 3-D grid with an exact
  kappa_2(B), and a symmetric random pattern made diagonally dominant.

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


def laplacian_csr(dims, kappa_b: float):
    """B = L + sigma I, L the Dirichlet 5-point (2-D) or 7-point (3-D) Laplacian
    on a grid of `dims` points in natural ordering, sigma chosen so that
    kappa_2(B) = kappa_b exactly (sigma may be negative; B stays SPD).
    Returns (row_ptr int64, col_idx int32, vals float64), columns ascending."""
    dims = tuple(int(d) for d in dims)
    m = int(np.prod(dims))
    lam_lo = sum(2.0 - 2.0 * np.cos(np.pi / (d + 1)) for d in dims)
    lam_hi = sum(2.0 - 2.0 * np.cos(d * np.pi / (d + 1)) for d in dims)
    sigma = (lam_hi - kappa_b * lam_lo) / (kappa_b - 1.0)
    strides = [int(np.prod(dims[a + 1:])) for a in range(len(dims))]
    idx = np.arange(m, dtype=np.int64)
    coord = [(idx // strides[a]) % dims[a] for a in range(len(dims))]
    offs, masks = [], []
    for a in range(len(dims)):  # -stride, largest stride first: ascending columns
        offs.append(-strides[a])
        masks.append(coord[a] > 0)
    offs.append(0)
    masks.append(np.ones(m, dtype=bool))
    for a in reversed(range(len(dims))):
        offs.append(strides[a])
        masks.append(coord[a] < dims[a] - 1)
    M = np.stack(masks, axis=1)
    cols = idx[:, None] + np.asarray(offs, dtype=np.int64)[None, :]
    vals = np.where(np.asarray(offs)[None, :] == 0, 2.0 * len(dims) + sigma, -1.0)
    vals = np.broadcast_to(vals, M.shape)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(M.sum(axis=1), out=row_ptr[1:])
    return row_ptr, cols[M].astype(np.int32), np.ascontiguousarray(vals[M], dtype=np.float64)


def random_spd_csr(m: int, per_row: int, kappa_b: float, seed: int):
    """Symmetric B with about 2*per_row off-diagonal entries per row at uniformly
    random columns (values uniform in [-1, 1]) and diagonal
    b_ii = sum_j |b_ij| + c, so that kappa_2(B) <= (2 max_i r_i + c) / c with
    r_i the off-diagonal row sums; c is set from kappa_b. Long-range pattern:
    the rows a sparse product gathers are scattered over the whole matrix."""
    rng = np.random.default_rng(seed)
    i = np.repeat(np.arange(m, dtype=np.int64), per_row)
    j = rng.integers(0, m, size=i.size)
    v = rng.uniform(-1.0, 1.0, size=i.size)
    keep = i != j
    i, j, v = i[keep], j[keep], v[keep]
    r = np.concatenate([i, j])
    c = np.concatenate([j, i])
    v = np.concatenate([v, v])
    key = r * m + c
    order = np.argsort(key, kind="stable")
    key, v = key[order], v[order]
    ukey, start = np.unique(key, return_index=True)
    v = np.add.reduceat(v, start)
    r, c = ukey // m, ukey % m
    rsum = np.zeros(m)
    np.add.at(rsum, r, np.abs(v))
    cdiag = 2.0 * rsum.max() / (kappa_b - 1.0)
    r = np.concatenate([r, np.arange(m, dtype=np.int64)])
    c = np.concatenate([c, np.arange(m, dtype=np.int64)])
    v = np.concatenate([v, rsum + cdiag])
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    np.cumsum(row_ptr, out=row_ptr)
    return row_ptr, c.astype(np.int32), v


def csr_to_dense(csr, m: int) -> np.ndarray:
    row_ptr, col_idx, vals = csr
    B = np.zeros((m, m))
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    np.add.at(B, (rows, col_idx.astype(np.int64)), vals)
    return B
