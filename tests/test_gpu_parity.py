"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Tolerances (FP64; both sides follow the same algorithm, so the differences
are rounding-order differences of the Gram sums, the FMA contraction and the
reciprocal in the substitution):
  * ||Q^T Q - I||_2 <= 1e-13 and ||X - QR||_F / ||X||_F <= 1e-13;
  * ||R_gpu - R_oracle||_F / ||R_oracle||_F <= 1e-12 for kappa_2(X) <= 1e8;
  * above that, R is compared with the bound c * kappa * u of its forward
    error (the factor is ill-conditioned in the same way for both sides).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1809_11085_gb300 import scqr3  # noqa: E402
from paper_1809_11085_gb300.testmat import (block_diag_spd, repeated_small_sigma,  # noqa: E402
                                            testmat)

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1809_11085_gb300 import build

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run_gpu(Xh, Bblk=None, **kw):
    X = torch.from_numpy(Xh).cuda()
    B = None if Bblk is None else torch.from_numpy(Bblk).cuda()
    Q, R, info = scqr3.factor(X, B, **kw)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), R.cpu().numpy(), info


def orth2(Q, Bblk=None):
    n = Q.shape[1]
    if Bblk is None:
        return np.linalg.norm(Q.T @ Q - np.eye(n), 2)
    bs = Bblk.shape[1]
    BQ = np.einsum("kij,kjn->kin", Bblk, Q.reshape(-1, bs, n)).reshape(Q.shape)
    return np.linalg.norm(Q.T @ BQ - np.eye(n), 2)


def resid(X, Q, R):
    return np.linalg.norm(X - Q @ R) / np.linalg.norm(X)


def check_pair(Xh, kappa, Bblk=None, orth_tol=1e-13, **kw):
    Qg, Rg, info = run_gpu(Xh, Bblk, **kw)
    Qo, Ro, st, tr = oracle.scqr3(Xh, Bblk, normx2=kw.get("norm_x2", 0.0), normb=kw.get("normb", 0.0),
                                  max_passes=kw.get("max_passes", 0) or 6)
    assert st == 0, (st, tr)
    assert info.status == 0, info
    n = Xh.shape[1]
    assert np.array_equal(np.tril(Rg, -1), np.zeros((n, n)))
    assert (np.diag(Rg) > 0).all()
    assert orth2(Qg, Bblk) <= orth_tol
    assert resid(Xh, Qg, Rg) <= 1e-13
    dR = np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro)
    if kappa <= 1e8:
        assert dR <= 1e-12, dR
    else:
        assert dR <= 100 * n * kappa * U, dR
    return Qg, Rg, info, Qo, Ro, tr


# ------------------------------------------------------------------------------- small workload (first config)

def test_first_config_20000x32_kappa_1e12():
    """X = U diag(sigma) V^T, 20000 x 32, sigma geometric 1 -> 1e-12."""
    Xh = testmat(20000, 32, 1e12, seed=1100)
    _, _, info, _, _, tr = check_pair(Xh, 1e12)
    assert info.shifted[0] == 1 and info.shifted[-2:] == [0, 0]


@pytest.mark.parametrize("kappa", [1e2, 1e5, 1e8])
def test_well_conditioned_R_matches_to_1e12(kappa):
    Xh = testmat(30000, 64, kappa, seed=1200 + int(np.log10(kappa)))
    _, _, info, _, _, tr = check_pair(Xh, kappa)
    # far from the breakdown threshold the pass sequences agree
    assert info.passes == tr["passes"] and info.shifted == tr["shifted"]
    assert info.s[0] == pytest.approx(tr["s"][0], rel=1e-12)


@pytest.mark.parametrize("n", [1, 2, 7, 16, 31, 32, 33, 63, 64, 100, 127, 128])
@pytest.mark.parametrize("m_kind", ["square", "plus1", "ragged", "tall"])
def test_shape_sweep(n, m_kind):
    m = {"square": n, "plus1": n + 1, "ragged": 97 * 7 + n, "tall": 4096 * 3 + 17}[m_kind]
    m = max(m, n)
    kappa = 1e6
    Xh = testmat(m, n, kappa, seed=1300 + n)
    check_pair(Xh, kappa)


@pytest.mark.parametrize("kappa", [1e10, 1e14, 1e15])
def test_ill_conditioned_extra_passes(kappa):
    Xh = testmat(50000, 32, kappa, seed=1400 + int(np.log10(kappa)))
    _, _, info, _, _, tr = check_pair(Xh, kappa)
    assert info.passes >= 3


def test_repeated_small_singular_values():
    n = 64
    Xh = testmat(40000, n, 0.0, seed=1500, sigma=repeated_small_sigma(n, 8, 1e-14, 1e7))
    Qg, Rg, info = run_gpu(Xh)
    assert info.status == 0
    assert orth2(Qg) <= 1e-13 and resid(Xh, Qg, Rg) <= 1e-13


def test_user_norm_x2_matches_paper_table1_shift():
    """With ||X||_2^2 = 1 given, pass 1 uses the shift of Eq. (finds2) exactly."""
    Xh = testmat(1000, 30, 1e12, seed=1600)
    Qg, Rg, info = run_gpu(Xh, norm_x2=1.0)
    assert info.s[0] == oracle.shift(1000, 30, 1.0)
    Qo, Ro, st, tr = oracle.scqr3(Xh, normx2=1.0)
    assert info.shifted == tr["shifted"]
    assert orth2(Qg) <= 1e-13


def test_in_place_and_leading_dimension():
    m, n = 5000, 24
    Xh = testmat(m, n, 1e9, seed=1700)
    wide = torch.zeros((m, n + 5), dtype=torch.float64, device="cuda")
    wide[:, 2:2 + n] = torch.from_numpy(Xh).cuda()
    Xv = wide[:, 2:2 + n]
    assert Xv.stride(0) == n + 5
    Q, R, info = scqr3.factor(Xv, Q=Xv)  # in place, ld = n + 5
    torch.cuda.synchronize()
    assert info.status == 0
    Qg = Q.cpu().numpy()
    Rg = R.cpu().numpy()
    assert orth2(Qg) <= 1e-13 and resid(Xh, Qg, Rg) <= 1e-13
    assert torch.all(wide[:, :2] == 0) and torch.all(wide[:, 2 + n:] == 0)
    Q2, R2, _ = run_gpu(Xh)
    assert np.array_equal(Q2, Qg) and np.array_equal(R2, Rg)


def test_deterministic():
    Xh = testmat(70000, 64, 1e12, seed=1800)
    a = run_gpu(Xh)
    b = run_gpu(Xh)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("kappa", [1e4, 1e13])
def test_rpass_product_is_R(kappa):
    m, n = 8000, 16
    Xh = testmat(m, n, kappa, seed=1900)
    X = torch.from_numpy(Xh).cuda()
    Rpass = torch.zeros((scqr3.MAX_PASSES, n, n), dtype=torch.float64, device="cuda")
    Q, R, info = scqr3.factor(X, Rpass=Rpass)
    torch.cuda.synchronize()
    Rp = Rpass.cpu().numpy()
    acc = np.eye(n)
    for k in range(info.passes):
        acc = Rp[k] @ acc
    assert np.linalg.norm(acc - R.cpu().numpy()) / np.linalg.norm(acc) < 1e-14
    if kappa > 1e6:
        return  # the replay below amplifies rounding-order differences by cond(R_1)
    # replay with the oracle's row solve: Q = X R_1^{-1} R_2^{-1} ... on sampled rows
    rows = np.arange(0, m, 97)
    Qs = Xh[rows]
    for k in range(info.passes):
        Qs = oracle.trsm(Qs, Rp[k])
    Qg = Q.cpu().numpy()[rows]
    assert np.max(np.abs(Qs - Qg)) < 1e3 * kappa * U * np.max(np.abs(Qg))


def test_status_codes():
    Xh = testmat(3000, 16, 1e4, seed=2000)
    Xh[17, 3] = np.nan
    _, _, info = run_gpu(Xh)
    assert info.status == scqr3.E_NONFINITE
    Xh = testmat(20000, 32, 1e15, seed=2001)
    _, _, info = run_gpu(Xh, max_passes=3)
    _, _, st, tr = oracle.scqr3(Xh, max_passes=3)
    if tr["passes"] == 3 and st == oracle.E_MAXPASS:
        assert info.status == scqr3.E_MAXPASS
    with pytest.raises(scqr3.ScqrError):
        scqr3.factor(torch.zeros((4, 8), dtype=torch.float64, device="cuda"))


# ------------------------------------------------------------------------------- oblique inner product

@pytest.mark.parametrize("bs", [1, 2, 4, 8, 16])
def test_oblique_block_sizes(bs):
    m, n = 4096, 32
    Bblk = block_diag_spd(m, bs, seed=2100 + bs)
    Xh = testmat(m, n, 1e6, seed=2200 + bs)
    check_pair(Xh, 1e6, Bblk)


@pytest.mark.parametrize("n", [16, 64, 128])
def test_oblique_config_shape(n):
    """B blocks G^T G + 0.1 I (8 x 8), kappa_2(X) = 1e10, shrunk m."""
    m = 32768
    Bblk = block_diag_spd(m, 8, seed=2300 + n)
    Xh = testmat(m, n, 1e10, seed=2400 + n)
    Qg, Rg, info = run_gpu(Xh, Bblk)
    assert info.status == 0, info
    assert orth2(Qg, Bblk) <= 1e-13
    assert resid(Xh, Qg, Rg) <= 1e-13
    _, Ro, st, tr = oracle.scqr3(Xh, Bblk)
    assert st == 0
    assert info.s[0] == pytest.approx(tr["s"][0], rel=1e-10)


def test_oblique_not_spd_block_is_reported():
    m, n = 256, 8
    Bblk = block_diag_spd(m, 8, seed=2500)
    Bblk[3] = -np.eye(8)
    _, _, info = run_gpu(testmat(m, n, 10.0, seed=2501), Bblk)
    assert info.status == scqr3.E_B_NOT_SPD


# ------------------------------------------------------------------------------- 128 < n <= 256

@pytest.mark.parametrize("n", [129, 200, 256])
@pytest.mark.parametrize("kappa", [1e4, 1e10])
def test_wide_n(n, kappa):
    m = 6000 + 37
    Xh = testmat(m, n, kappa, seed=2600 + n)
    check_pair(Xh, kappa)


def test_wide_n_square_and_rejections():
    Xh = testmat(256, 256, 1e6, seed=2700)
    check_pair(Xh, 1e6)
    X = torch.zeros((1024, 200), dtype=torch.float64, device="cuda")
    with pytest.raises(scqr3.ScqrError):
        scqr3.factor(X, precision=scqr3.PREC_MIXED)
    with pytest.raises(scqr3.ScqrError):
        scqr3.factor(torch.zeros((1024, 257), dtype=torch.float64, device="cuda"))
