"""GPU parity of the oblique inner product with a sparse SPD B in CSR form
(Alg. 5 with the sparse product B Q of Sec. 7.2) against the oracle.

Inputs stand in for the paper's SuiteSparse matrices (not available): the
shifted Dirichlet Laplacian of a 2-D or 3-D grid with exact kappa_2(B), and a
diagonally dominant random pattern whose rows reach across the whole matrix.

Tolerances: ||Q^T B Q - I||_2 <= 1e-12 and ||X - QR||_F / ||X||_F <= 1e-13,
as for the block-diagonal B; R against the oracle within
100 n kappa(X) sqrt(kappa(B)) u, the forward-error scale of the R factor of
L^T X (B = L L^T). The device sums the Gram matrix in another order and, for
the pairs past the diagonal of its cyclic layout, uses (Y^T Q)_{kj} for
(Q^T Y)_{kj} (equal in exact arithmetic, B symmetric).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1809_11085_gb300 import scqr3  # noqa: E402
from paper_1809_11085_gb300.testmat import (block_diag_spd, laplacian_csr,  # noqa: E402
                                            random_spd_csr, testmat)

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1809_11085_gb300 import build

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def bq(csr, Q):
    """B Q on the host from the CSR arrays (plain numpy, for checking only)."""
    row_ptr, col_idx, vals = csr
    m = len(row_ptr) - 1
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    out = np.zeros_like(Q)
    np.add.at(out, rows, vals[:, None] * Q[col_idx.astype(np.int64)])
    return out


def run(Xh, csr, **kw):
    X = torch.from_numpy(Xh).cuda()
    B = scqr3.CsrB.from_arrays(csr)
    Q, R, info = scqr3.factor(X, B, **kw)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), R.cpu().numpy(), info


def check(Xh, csr, kappa_x, kappa_b, oracle_kw=None, **kw):
    Qg, Rg, info = run(Xh, csr, **kw)
    okw = dict(normx2=kw.get("norm_x2", 0.0), shift_scale=kw.get("shift_scale", 0.0),
               algorithm=kw.get("algorithm", 3), max_passes=kw.get("max_passes", 0) or 6)
    okw.update(oracle_kw or {})
    Qo, Ro, st, tr = oracle.scqr3(Xh, csr=csr, **okw)
    assert st == 0 and info.status == 0, (st, info)
    assert info.passes == tr["passes"] and info.shifted[:info.passes] == tr["shifted"]
    n = Xh.shape[1]
    assert np.array_equal(np.tril(Rg, -1), np.zeros((n, n)))
    assert (np.diag(Rg) > 0).all()
    assert np.linalg.norm(Qg.T @ bq(csr, Qg) - np.eye(n), 2) <= 1e-12
    assert np.linalg.norm(Xh - Qg @ Rg) / np.linalg.norm(Xh) <= 1e-13
    dR = np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro)
    assert dR <= max(1e-12, 100 * n * kappa_x * np.sqrt(kappa_b) * U), dR
    return info, tr


@pytest.mark.parametrize("n", [1, 7, 16, 32, 33, 64, 100, 128])
def test_laplacian_2d(n):
    csr = laplacian_csr((100, 121), 1e3)
    Xh = testmat(12100, n, 1e10, seed=4000 + n)
    info, tr = check(Xh, csr, 1e10, 1e3, norm_x2=1.0)
    # same ||B|| bound (largest absolute row sum, same order) and ||X|| => same shift
    assert info.s[0] == tr["s"][0]


@pytest.mark.parametrize("n", [16, 64, 128])
@pytest.mark.parametrize("kappa,passes", [(1e9, 3), (1e14, 4)])
def test_laplacian_3d_ragged(n, kappa, passes):
    """12673 rows: no panel size divides it. kappa(X) = 1e14 needs a second
    shifted pass (the Gram of Q1 is indefinite in the oracle), 1e9 does not."""
    csr = laplacian_csr((19, 23, 29), 1e2)
    Xh = testmat(12673, n, kappa, seed=4100 + n)
    info, tr = check(Xh, csr, kappa, 1e2)
    assert tr["passes"] == passes


@pytest.mark.parametrize("n", [32, 64])
def test_random_long_range_pattern(n):
    csr = random_spd_csr(9000, 3, 1e3, seed=4200 + n)
    Xh = testmat(9000, n, 1e8, seed=4201 + n)
    check(Xh, csr, 1e8, 1e3)


def test_block_diagonal_as_csr_matches_both_forms():
    """The block-diagonal B of the oblique benchmark, stored as CSR: the CSR
    path and the block path (Z = L^T Q) agree with each other and the oracle."""
    m, n, bs = 8192, 32, 8
    Bblk = block_diag_spd(m, bs, seed=4300)
    rows, cols, vals = [], [], []
    for k in range(m // bs):
        r, c = np.meshgrid(np.arange(bs) + k * bs, np.arange(bs) + k * bs, indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(Bblk[k].ravel())
    rows = np.concatenate(rows)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    csr = (np.cumsum(row_ptr), np.concatenate(cols).astype(np.int32), np.concatenate(vals))
    Xh = testmat(m, n, 1e10, seed=4301)
    nb = float(oracle.normb_bound(Bblk))
    Qc, Rc, ic = run(Xh, csr, normb=nb)
    Qb, Rb, ib = scqr3.factor(torch.from_numpy(Xh).cuda(), torch.from_numpy(Bblk).cuda(), normb=nb)
    assert ic.status == 0 and ib.status == 0
    Rb = Rb.cpu().numpy()
    assert np.linalg.norm(Rc - Rb) / np.linalg.norm(Rb) < 100 * n * 1e10 * np.sqrt(1e3) * U
    check(Xh, csr, 1e10, 1e3, normb=nb, oracle_kw={"normb": nb})


def test_alg2_and_small_shift_with_csr():
    """kappa(Q1)^2 u is 1e-4 (Alg. 2, kappa(X) = 1e10) and 1e-5 (c = 500,
    kappa(X) = 1e12), and the smaller shift is 400x the Gram's negative noise
    eigenvalue: no pass decision is near its threshold."""
    csr = laplacian_csr((64, 64), 1e3)
    check(testmat(4096, 48, 1e10, seed=4400), csr, 1e10, 1e3, norm_x2=1.0,
          algorithm=scqr3.ALG_ADAPTIVE)
    info, tr = check(testmat(4096, 48, 1e12, seed=4400), csr, 1e12, 1e3, norm_x2=1.0,
                     shift_scale=500.0)
    assert info.s[0] == tr["s"][0]


def test_deterministic_and_in_place():
    csr = laplacian_csr((80, 80), 1e3)
    Xh = testmat(6400, 64, 1e10, seed=4500)
    Q1, R1, _ = run(Xh, csr)
    Q2, R2, _ = run(Xh, csr)
    assert np.array_equal(Q1, Q2) and np.array_equal(R1, R2)
    X = torch.from_numpy(Xh).cuda()
    Q, R, info = scqr3.factor(X, scqr3.CsrB.from_arrays(csr), Q=X)
    torch.cuda.synchronize()
    assert info.status == 0
    assert np.array_equal(X.cpu().numpy(), Q1) and np.array_equal(R.cpu().numpy(), R1)


@pytest.mark.parametrize("defect", ["column_out_of_range", "no_diagonal", "row_ptr_decreasing",
                                    "row_ptr_past_nnz", "negative_diagonal"])
def test_malformed_csr_is_reported(defect):
    """Every range and index the kernels read is clamped to the arrays, so a
    malformed B is reported (SCQR3_E_B_INVALID) instead of read out of bounds."""
    rp, ci, v = (a.copy() for a in laplacian_csr((30, 40), 1e2))
    m = len(rp) - 1
    if defect == "column_out_of_range":
        ci[17] = m + 5
    elif defect == "no_diagonal":
        r = 100
        d = rp[r] + int(np.nonzero(ci[rp[r]:rp[r + 1]] == r)[0][0])
        ci[d] = (r + 7) % m
    elif defect == "row_ptr_decreasing":
        rp[200] = rp[202] + 1
    elif defect == "row_ptr_past_nnz":
        rp[m] = rp[m] + 1000
    else:
        r = 300
        d = rp[r] + int(np.nonzero(ci[rp[r]:rp[r + 1]] == r)[0][0])
        v[d] = -v[d]
    Xh = testmat(m, 8, 1e4, seed=4600)
    _, _, info = run(Xh, (rp, ci, v))
    assert info.status == scqr3.E_B_INVALID


def test_large_laplacian_properties():
    """1,048,576 rows (1024 x 1024 grid), n = 128: properties at a size the
    oracle cannot finish quickly; B Q by torch's sparse product, for checking."""
    csr = laplacian_csr((1024, 1024), 1e3)
    m, n = 1024 * 1024, 128
    from paper_1809_11085_gb300.testmat import testmat_torch

    X, _, _ = testmat_torch(m, n, 1e10, seed=4700)
    B = scqr3.CsrB.from_arrays(csr)
    Q, R, info = scqr3.factor(X, B)
    torch.cuda.synchronize()
    assert info.status == 0 and info.passes == 3
    Bt = torch.sparse_csr_tensor(B.row_ptr, B.col_idx.to(torch.int64), B.vals, size=(m, m))
    G = Q.T @ (Bt @ Q)
    assert torch.linalg.matrix_norm(G - torch.eye(n, dtype=torch.float64, device="cuda"), 2) < 1e-12
    assert torch.linalg.matrix_norm(X - Q @ R) / torch.linalg.matrix_norm(X) < 1e-13
