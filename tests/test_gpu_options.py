"""GPU parity of the two options beyond Alg. 3: the smaller first shift of the
remark in Sec. 6.1 (scqr3_opts.shift_scale) and the adaptive Alg. 2
(scqr3_opts.algorithm / tol), each against the oracle run with the same
options.

Decisions (which shift, how many passes) are compared only where they are not
marginal: the margin between the shifted Gram's smallest eigenvalue and zero,
or between ||Q^T Q - I||_F and the tolerance, is at least a factor of 4 in
every case below, so rounding-order differences of the Gram sums cannot flip
them. Values use the tolerances of the Alg. 3 parity tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1809_11085_gb300 import scqr3  # noqa: E402
from paper_1809_11085_gb300.testmat import block_diag_spd, testmat  # noqa: E402

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


def compare(Xh, kappa, Qg, Rg, info, Qo, Ro, st, tr, orth_tol=1e-13, Bblk=None):
    assert st == 0 and info.status == 0, (st, info)
    assert info.passes == tr["passes"]
    assert info.shifted[:info.passes] == tr["shifted"]
    n = Xh.shape[1]
    assert np.array_equal(np.tril(Rg, -1), np.zeros((n, n)))
    assert (np.diag(Rg) > 0).all()
    assert orth2(Qg, Bblk) <= orth_tol
    assert resid(Xh, Qg, Rg) <= 1e-13
    dR = np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro)
    assert dR <= (1e-12 if kappa <= 1e8 else 100 * n * kappa * U), dR


# ------------------------------------------------------------------------------- smaller shift

@pytest.mark.parametrize("m,n,kappa,c", [(1000, 50, 1e15, 10.0), (60000, 64, 1e14, 1e3),
                                         (20000, 128, 1e14, 1e3), (3000, 200, 1e14, 1e3)])
def test_small_shift_saves_a_pass(m, n, kappa, c):
    """Sec. 6.1 remark (first case: its Fig. 3 setup): s = c u ||X||^2 succeeds
    and CholeskyQR2 finishes (3 passes), where the safe shift needs 4. c is
    chosen so that s is at least 5x the Gram's rounding noise and
    kappa(Q1)^2 = s kappa^2 is 8x below 1/u."""
    Xh = testmat(m, n, kappa, seed=2100 + n)
    Qg, Rg, info = run_gpu(Xh, norm_x2=1.0, shift_scale=c)
    Qo, Ro, st, tr = oracle.scqr3(Xh, normx2=1.0, shift_scale=c)
    assert tr["passes"] == 3
    assert info.s[0] == tr["s"][0] == c * U
    compare(Xh, kappa, Qg, Rg, info, Qo, Ro, st, tr)
    _, _, info_safe = run_gpu(Xh, norm_x2=1.0)
    assert info_safe.passes == 4 and info_safe.shifted[:4] == [1, 1, 0, 0]


def test_small_shift_mixed_precision():
    Xh = testmat(40000, 64, 1e10, seed=2200)
    Qg, Rg, info = run_gpu(Xh, norm_x2=1.0, shift_scale=1e4, precision=scqr3.PREC_MIXED)
    Qo, Ro, st, tr = oracle.scqr3(Xh, normx2=1.0, shift_scale=1e4)
    assert info.s[0] == 1e4 * U
    compare(Xh, 1e10, Qg, Rg, info, Qo, Ro, st, tr, orth_tol=1e-13)


@pytest.mark.parametrize("n", [32, 128, 256])
def test_small_shift_falls_back_to_safe_shift(n):
    """s = 1e-6 u ||X||^2 is far below the rounding error of the computed Gram
    matrix, whose ~n/2 noise-level eigenvalues (kappa 1e15) are then certain to
    include negative ones: the Cholesky breaks down and the shift of
    Eq. (finds2) follows, so the run is bit for bit the default one."""
    Xh = testmat(4 * n + 7, n, 1e15, seed=2300 + n)
    Qa, Ra, ia = run_gpu(Xh, shift_scale=1e-6)
    Qb, Rb, ib = run_gpu(Xh)
    assert ia.status == 0 and ib.status == 0
    assert ia.s[:ia.passes] == ib.s[:ib.passes]
    assert abs(ia.s[0] / oracle.shift(Xh.shape[0], n, float((Xh * Xh).sum())) - 1) < 1e-12
    assert np.array_equal(Qa, Qb) and np.array_equal(Ra, Rb)


def test_small_shift_oblique():
    m, n, bs = 4096, 32, 8
    Bblk = block_diag_spd(m, bs, seed=2401)
    Xh = testmat(m, n, 1e10, seed=2402)
    Qg, Rg, info = run_gpu(Xh, Bblk, norm_x2=1.0, normb=float(oracle.normb_bound(Bblk)),
                           shift_scale=1e4)
    Qo, Ro, st, tr = oracle.scqr3(Xh, Bblk, normx2=1.0, normb=oracle.normb_bound(Bblk),
                                  shift_scale=1e4)
    assert info.s[0] == tr["s"][0]
    compare(Xh, 1e10, Qg, Rg, info, Qo, Ro, st, tr, orth_tol=1e-12, Bblk=Bblk)


# ------------------------------------------------------------------------------- Alg. 2

@pytest.mark.parametrize("m,n,kappa", [(1000, 30, 1e12), (100, 100, 1e13), (200000, 64, 1e11),
                                       (30000, 128, 1e11), (5000, 160, 1e11), (20000, 16, 1e12)])
def test_alg2_table_setups(m, n, kappa):
    """Tables 1-2: Alg. 2's plain Cholesky of X^T X breaks down, one shifted
    pass and two plain passes follow, and the stopping test ends the loop."""
    Xh = testmat(m, n, kappa, seed=2500 + n)
    Qg, Rg, info = run_gpu(Xh, norm_x2=1.0, algorithm=scqr3.ALG_ADAPTIVE)
    Qo, Ro, st, tr = oracle.scqr3(Xh, normx2=1.0, algorithm=2)
    assert tr["passes"] == 3 and tr["shifted"] == [1, 0, 0]
    assert info.unshifted_fail[0] > 0 and info.unshifted_fail[1:3] == [0, 0]
    compare(Xh, kappa, Qg, Rg, info, Qo, Ro, st, tr)


@pytest.mark.parametrize("n", [16, 64, 128, 200])
@pytest.mark.parametrize("kappa,passes", [(1.0, 1), (1e5, 2)])
def test_alg2_well_conditioned_needs_no_shift(n, kappa, passes):
    m = 50 * n + 3
    Xh = testmat(m, n, kappa, seed=2600 + n)
    Qg, Rg, info = run_gpu(Xh, algorithm=scqr3.ALG_ADAPTIVE)
    Qo, Ro, st, tr = oracle.scqr3(Xh, algorithm=2)
    assert tr["passes"] == passes and tr["shifted"] == [0] * passes
    compare(Xh, kappa, Qg, Rg, info, Qo, Ro, st, tr)


@pytest.mark.parametrize("kappa", [1e11, 1.0])
def test_alg2_mixed_precision(kappa):
    """The mixed form keeps iterates as float pairs until its last solve; under
    Alg. 2 every solve is followed by a Gram step, so the stop leaves pairs that
    the finishing kernel turns into FP64 Q."""
    Xh = testmat(100000, 64, kappa, seed=2700)
    Qg, Rg, info = run_gpu(Xh, norm_x2=1.0, algorithm=scqr3.ALG_ADAPTIVE, precision=scqr3.PREC_MIXED)
    Qo, Ro, st, tr = oracle.scqr3(Xh, normx2=1.0, algorithm=2)
    assert tr["passes"] == (3 if kappa > 1 else 1)
    compare(Xh, kappa, Qg, Rg, info, Qo, Ro, st, tr)


def test_alg2_oblique():
    m, n, bs = 4096, 32, 4
    Bblk = block_diag_spd(m, bs, seed=2801)
    Xh = testmat(m, n, 1e9, seed=2802)
    Qg, Rg, info = run_gpu(Xh, Bblk, algorithm=scqr3.ALG_ADAPTIVE)
    Qo, Ro, st, tr = oracle.scqr3(Xh, Bblk, algorithm=2)
    compare(Xh, 1e9, Qg, Rg, info, Qo, Ro, st, tr, orth_tol=1e-12, Bblk=Bblk)


@pytest.mark.parametrize("n", [30, 200])
def test_alg2_printed_tolerance_runs_to_the_pass_limit(n):
    """With tol = sqrt(n) u the test is never met on a computed Gram matrix:
    every allowed pass runs and the status is SCQR3_E_MAXPASS, as in the
    oracle; the factorization itself is complete and accurate."""
    Xh = testmat(1000, n, 1e12, seed=2900 + n)
    tol = np.sqrt(n) * U
    Qg, Rg, info = run_gpu(Xh, norm_x2=1.0, algorithm=scqr3.ALG_ADAPTIVE, tol=tol, max_passes=5)
    _, _, st, tr = oracle.scqr3(Xh, normx2=1.0, algorithm=2, tol=tol, max_passes=5)
    assert st == oracle.E_MAXPASS and tr["passes"] == 5
    assert info.status == scqr3.E_MAXPASS and info.passes == 5
    assert orth2(Qg) < 1e-13 and resid(Xh, Qg, Rg) < 1e-13


def test_alg2_rpass_and_backward_consistent():
    """The per-pass factors of an Alg. 2 run multiply to R, and the pass-wise
    adjoint accepts its pass count (two passes here)."""
    Xh = testmat(20000, 32, 1e4, seed=3001)
    X = torch.from_numpy(Xh).cuda()
    Rpass = torch.zeros((scqr3.MAX_PASSES, 32, 32), dtype=torch.float64, device="cuda")
    Q, R, info = scqr3.factor(X, algorithm=scqr3.ALG_ADAPTIVE, Rpass=Rpass)
    assert info.status == 0 and info.passes == 2
    Rp = Rpass.cpu().numpy()
    assert np.linalg.norm(Rp[1] @ Rp[0] - R.cpu().numpy()) / np.linalg.norm(Rp[0]) < 1e-14
    dQ = torch.randn_like(Q)
    dX = scqr3.backward(Q, Rpass, info.passes, dQ)
    torch.cuda.synchronize()
    from oracle.adjoint import qr_adjoint

    ref = qr_adjoint(Q.cpu().numpy(), R.cpu().numpy(), dQ.cpu().numpy(), np.zeros((32, 32)))
    assert np.linalg.norm(dX.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-10


def test_option_rejections():
    X = torch.from_numpy(testmat(100, 4, 10.0, seed=3101)).cuda()
    with pytest.raises(scqr3.ScqrError):
        scqr3.factor(X, algorithm=1)
    with pytest.raises(scqr3.ScqrError):
        scqr3.factor(X, algorithm=4)


@pytest.mark.parametrize("m,n", [(20000, 64), (3000, 128), (2000, 200)])
@pytest.mark.parametrize("algorithm", [scqr3.ALG_ADAPTIVE, scqr3.ALG_SCQR3])
def test_beyond_one_over_u(m, n, algorithm):
    """kappa(X) = 1e18 > 1/u (Sec. 4: Alg. 2 may still work). The pass count is
    not compared (it depends on where rounding puts the noise eigenvalues);
    the bounds of Thm. (maincholqr3) are."""
    Xh = testmat(m, n, 1e18, seed=3200 + n)
    Qg, Rg, info = run_gpu(Xh, norm_x2=1.0, algorithm=algorithm, max_passes=8)
    assert info.status == 0 and info.passes >= 4
    k = info.passes
    assert info.shifted[:k] == [1] * (k - 2) + [0, 0]
    assert np.linalg.norm(Qg.T @ Qg - np.eye(n)) <= 6 * (m * n + n * (n + 1)) * U
    assert np.linalg.norm(Qg @ Rg - Xh) / np.linalg.norm(Xh, 2) <= 15 * n * n * U
    assert (np.diag(Rg) > 0).all()


@pytest.mark.parametrize("precision", [scqr3.PREC_FP64, scqr3.PREC_TC])
@pytest.mark.parametrize("m,n,kappa", [(20000, 32, 1e12), (30011, 64, 1e15), (5000, 100, 1e8)])
def test_two_norm_estimate_shift(precision, m, n, kappa):
    """norm_x2 = SCQR3_NORM_X2_TWO_EST: every shifted pass estimates ||Q||_2^2
    as lambda_max of its Gram matrix by the power method (Sec. 4.1, normest),
    on the device as in the oracle: the estimates and shifts agree to 1e-10
    (the Gram matrices differ only by rounding), the first is ||X||_2^2 = 1 of
    the construction, and the results meet the FP64 tolerances."""
    Xh = testmat(m, n, kappa, seed=7700 + n)
    Q, R, info = scqr3.factor(torch.from_numpy(Xh).cuda(), norm_x2=scqr3.NORM_X2_TWO_EST, precision=precision)
    torch.cuda.synchronize()
    Qo, Ro, st, tr = oracle.scqr3(Xh, normx2=oracle.TWO_NORM_EST)
    assert st == 0 and info.status == 0, info
    assert abs(info.norm2[0] - 1.0) <= 1e-10 and abs(tr["norm2"][0] - 1.0) <= 1e-10
    for p in range(min(info.passes, tr["passes"])):
        if info.shifted[p] and tr["shifted"][p]:
            assert abs(info.s[p] - tr["s"][p]) <= 1e-9 * tr["s"][p], (p, info.s[p], tr["s"][p])
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    assert np.linalg.norm(Q.T @ Q - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(Xh - Q @ R) / np.linalg.norm(Xh) <= 1e-13
    dR = np.linalg.norm(R - Ro) / np.linalg.norm(Ro)
    assert dR <= (1e-12 if kappa <= 1e8 else 100 * n * kappa * U), dR


def test_two_norm_estimate_rejected_with_b():
    from paper_1809_11085_gb300.testmat import block_diag_spd

    X = torch.zeros((800, 16), dtype=torch.float64, device="cuda")
    B = torch.from_numpy(block_diag_spd(800, 8, seed=1)).cuda()
    with pytest.raises(scqr3.ScqrError) as e:
        scqr3.factor(X, B, norm_x2=scqr3.NORM_X2_TWO_EST)
    assert e.value.code == -12
