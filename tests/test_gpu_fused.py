"""GPU parity of the one-sweep tensor-core substitution (SCQR3_PREC_TC,
16 < n <= 64): each pass reads every row once, solves its 16-column diagonal
blocks in FP64 with the row in registers, applies the off-diagonal blocks of
R_k on the tensor cores (exact digit split), writes the row once and hands the
column maxima of the result to the next tensor-core Gram matrix.

Tolerances are the FP64 parity tolerances against the oracle (the split's
error is a perturbation of R of norm O(u ||R||) per row, the form of the
row-wise backward error that Sec. 3 assumes): ||Q^T Q - I||_2 <= 1e-13,
||X - QR||_F / ||X||_F <= 1e-13, R within 1e-12 (kappa <= 1e8) or
100 n kappa u. The same inputs also go through the separate-launch form
(scqr3_debug_set(SCQR3_DEBUG_FUSED_SOLVE, 0)) for comparison.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1809_11085_gb300 import scqr3  # noqa: E402
from paper_1809_11085_gb300.testmat import testmat  # noqa: E402

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
TC = scqr3.PREC_TC


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1809_11085_gb300 import build

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    scqr3.debug_set(scqr3.DEBUG_FUSED_SOLVE, 1)
    scqr3.debug_set(scqr3.DEBUG_WAIT_NS, -1)


def run(Xh, fused=True, **kw):
    scqr3.debug_set(scqr3.DEBUG_FUSED_SOLVE, 1 if fused else 0)
    try:
        Q, R, info = scqr3.factor(torch.from_numpy(Xh).cuda(), precision=TC, **kw)
        torch.cuda.synchronize()
    finally:
        scqr3.debug_set(scqr3.DEBUG_FUSED_SOLVE, 1)
    return Q.cpu().numpy(), R.cpu().numpy(), info


def check_against_oracle(Xh, kappa, Qg, Rg, info, **kw):
    Qo, Ro, st, tr = oracle.scqr3(Xh, normx2=kw.get("norm_x2", 0.0), algorithm=kw.get("algorithm", 3))
    assert st == 0 and info.status == 0, (st, info)
    n = Xh.shape[1]
    assert np.array_equal(np.tril(Rg, -1), np.zeros((n, n)))
    assert (np.diag(Rg) > 0).all()
    assert np.linalg.norm(Qg.T @ Qg - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(Xh - Qg @ Rg) / np.linalg.norm(Xh) <= 1e-13
    dR = np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro)
    assert dR <= (1e-12 if kappa <= 1e8 else 100 * n * kappa * U), dR
    return tr


@pytest.mark.parametrize("n", [17, 24, 31, 32, 33, 40, 48, 63, 64])
@pytest.mark.parametrize("m_kind", ["square", "tiny", "one_tile", "ragged", "tall"])
def test_fused_shape_sweep(n, m_kind):
    """NP = 32 (n <= 32: one update) and NP = 64 (three updates, the middle one
    with K = 32); m from n to several hundred tiles, ragged last tile, fewer
    rows than one tile, and fewer tiles than CTA slots."""
    m = {"square": n, "tiny": 100, "one_tile": 128, "ragged": 20011, "tall": 100003}[m_kind]
    m = max(m, n)
    kappa = 1e6
    Xh = testmat(m, n, kappa, seed=9000 + 7 * n + m)
    Qf, Rf, inf = run(Xh)
    check_against_oracle(Xh, kappa, Qf, Rf, inf)
    Qs, Rs, ins = run(Xh, fused=False)
    assert ins.status == 0 and ins.passes == inf.passes
    assert np.linalg.norm(Rf - Rs) / np.linalg.norm(Rs) <= 1e-12


@pytest.mark.parametrize("scale", [0.0, 1e-9, 1e-3])
def test_rows_with_a_small_leading_block(scale):
    """The middle product uses one scale per row for y_0 and y_1; the first
    product's scale, taken with headroom from y_0 alone, serves both unless y_1
    is larger, and those rows cut y_0 again. Rows whose leading 16 entries are
    zero or far below the rest take that second path (every 3rd and 7th row
    here, so that most warps hold both kinds of row)."""
    m, n, kappa = 60013, 64, 1e6
    Xh = testmat(m, n, kappa, seed=9400)
    Xh[::3, :16] *= scale
    Xh[::7, :16] = 0.0
    Qf, Rf, inf = run(Xh)
    Qo, Ro, st, tr = oracle.scqr3(Xh)
    assert st == 0 and inf.status == 0, (st, inf)
    assert np.linalg.norm(Qf.T @ Qf - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(Xh - Qf @ Rf) / np.linalg.norm(Xh) <= 1e-13
    kx = np.linalg.cond(Xh)
    dR = np.linalg.norm(Rf - Ro) / np.linalg.norm(Ro)
    assert dR <= max(1e-12, 100 * n * kx * U), (dR, kx)


@pytest.mark.parametrize("kappa", [1e2, 1e8, 1e12, 1e15])
@pytest.mark.parametrize("n", [32, 64])
def test_fused_conditioning(n, kappa):
    Xh = testmat(60000, n, kappa, seed=9100 + n)
    Qf, Rf, inf = run(Xh, norm_x2=1.0)
    tr = check_against_oracle(Xh, kappa, Qf, Rf, inf, norm_x2=1.0)
    if kappa in (1e2, 1e8):
        assert inf.passes == tr["passes"] == 3


def test_fused_deterministic_in_place_and_leading_dimension():
    """Two calls give the same bits; in place (Q = X) with ld > n and a
    separate Q with its own ld give the same bits, and the columns around the
    views stay untouched."""
    m, n = 50001, 48
    Xh = testmat(m, n, 1e9, seed=9200)
    Q1, R1, i1 = run(Xh)
    Q2, R2, i2 = run(Xh)
    assert np.array_equal(Q1, Q2) and np.array_equal(R1, R2)
    wide = torch.zeros((m, n + 5), dtype=torch.float64, device="cuda")
    wide[:, 2:2 + n] = torch.from_numpy(Xh).cuda()
    Xv = wide[:, 2:2 + n]
    outw = torch.full((m, n + 3), 7.0, dtype=torch.float64, device="cuda")
    Qv = outw[:, 1:1 + n]
    Qa, Ra, ia = scqr3.factor(torch.from_numpy(Xh).cuda(), Q=Qv, precision=TC)
    Qb, Rb, ib = scqr3.factor(Xv, Q=Xv, precision=TC)
    torch.cuda.synchronize()
    assert ia.status == 0 and ib.status == 0
    assert torch.equal(Qa, Qb) and torch.equal(Ra, Rb)
    assert np.array_equal(Qa.cpu().numpy(), Q1) and np.array_equal(Ra.cpu().numpy(), R1)
    assert torch.all(wide[:, :2] == 0) and torch.all(wide[:, 2 + n:] == 0)
    assert torch.all(outw[:, :1] == 7.0) and torch.all(outw[:, 1 + n:] == 7.0)


def test_fused_column_maxima_feed_the_gram():
    """Columns scaled from 2^-200 to 2^200 and rows spanning 1e-30 .. 1: the
    next Gram matrix takes its column scales from the maxima the substitution
    emitted, so they must be exact; the result matches the FP64 form."""
    rng = np.random.default_rng(9300)
    m, n = 30000, 40
    Xh = testmat(m, n, 1e4, seed=9301)
    Xh *= np.exp2(rng.integers(-200, 200, size=n))[None, :]
    Xh[rng.random(m) < 0.3] *= 1e-30
    Qg, Rg, info = run(Xh)
    assert info.status == 0
    Qd, Rd, idv = scqr3.factor(torch.from_numpy(Xh).cuda())
    Rd = Rd.cpu().numpy()
    assert info.passes == idv.passes
    scale = np.abs(np.diag(Rd))
    assert np.linalg.norm((Rg - Rd) / scale[None, :]) < 1e-10
    assert np.linalg.norm(Qg.T @ Qg - np.eye(n), 2) < 1e-13


def test_fused_non_finite():
    for n, (i, j, v) in ((40, (777, 39, np.inf)), (64, (12345, 17, np.nan)), (20, (5, 0, -np.inf))):
        Xh = testmat(20000, n, 1e4, seed=9400 + n)
        Xh[i, j] = v
        _, _, info = run(Xh)
        assert info.status == scqr3.E_NONFINITE, (n, info)


def test_fused_host_form_chunks():
    """factor_host solves the last pass in row chunks (each one launch of the
    one-sweep kernel over its rows): one chunk gives the device call's bits;
    three chunks are held to the FP64 tolerances."""
    n = 64
    for m, seed in ((200000, 9500), (600000, 9501)):
        Xh = testmat(m, n, 1e10, seed=seed)
        Qd, Rd, idv = run(Xh)
        X = torch.empty(Xh.shape, dtype=torch.float64, pin_memory=True)
        X.copy_(torch.from_numpy(Xh))
        Qh, Rh, ih = scqr3.factor_host(X, precision=TC)
        Qh, Rh = Qh.numpy(), Rh.numpy()
        assert ih.status == 0 and idv.status == 0
        if m <= 262144:
            assert np.array_equal(Qh, Qd) and np.array_equal(Rh, Rd)
        else:
            assert np.linalg.norm(Qh.T @ Qh - np.eye(n), 2) <= 1e-13
            assert np.linalg.norm(Xh - Qh @ Rh) / np.linalg.norm(Xh) <= 1e-13
            assert np.linalg.norm(Rh - Rd) / np.linalg.norm(Rd) <= 100 * n * 1e10 * U


def test_fused_alg2_small_shift_and_oblique():
    """Alg. 2, the smaller first shift and a block-diagonal B (the oblique
    Gram scans Z = L^T Q itself) go through the same substitution."""
    from paper_1809_11085_gb300.testmat import block_diag_spd

    Xh = testmat(60000, 56, 1e5, seed=9600)
    Qa, Ra, ia = run(Xh, algorithm=scqr3.ALG_ADAPTIVE)
    check_against_oracle(Xh, 1e5, Qa, Ra, ia, algorithm=scqr3.ALG_ADAPTIVE)
    Qs, Rs, isv = run(testmat(60000, 64, 1e7, seed=9601), shift_scale=500.0)
    assert isv.status == 0
    assert np.linalg.norm(Qs.T @ Qs - np.eye(64), 2) <= 1e-13
    m, n, bs = 24000, 64, 8
    Xh = testmat(m, n, 1e8, seed=9602)
    Bh = block_diag_spd(m, bs, seed=9603)
    Q, R, info = scqr3.factor(torch.from_numpy(Xh).cuda(), torch.from_numpy(Bh).cuda(), precision=TC)
    torch.cuda.synchronize()
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    Qo, Ro, st, tr = oracle.scqr3(Xh, Bblk=Bh)
    assert st == 0 and info.status == 0 and info.passes == tr["passes"]
    BQ = np.einsum("kij,kjn->kin", Bh, Q.reshape(-1, bs, n)).reshape(Q.shape)
    assert np.linalg.norm(Q.T @ BQ - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-12


def exact_r(s, V):
    """R factor (positive diagonal) of diag(s) V^T: the exact R of
    X = U diag(s) V^T for orthonormal U, independent of m."""
    _, Re = np.linalg.qr(np.diag(s) @ V.T)
    return Re * np.sign(np.diag(Re))[:, None]


@pytest.mark.parametrize("kappa", [1e4, 1e8])
def test_fused_4m_rows_against_exact_r(kappa):
    """4,194,304 x 64 against the m-independent exact R (the R factor of
    Sigma V^T; U is orthonormal to about 1e-15 and moves R by that much
    relatively), and against the FP64 DFMA form, at the FP64 tolerances."""
    from paper_1809_11085_gb300.testmat import testmat_torch

    m, n = 4_194_304, 64
    X, s, V = testmat_torch(m, n, kappa, seed=9700 + int(np.log10(kappa)))
    Re = exact_r(s.cpu().numpy(), V.cpu().numpy())
    Qt, Rt, it = scqr3.factor(X, precision=TC)
    torch.cuda.synchronize()
    assert it.status == 0 and it.passes == 3
    Rth = Rt.cpu().numpy()
    assert np.linalg.norm(Rth - Re) / np.linalg.norm(Re) <= 1e-12
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    assert torch.linalg.matrix_norm(Qt.T @ Qt - eye, 2).item() <= 1e-13
    assert (torch.linalg.matrix_norm(X - Qt @ Rt) / torch.linalg.matrix_norm(X)).item() <= 1e-13
    del Qt
    Qd, Rd, idv = scqr3.factor(X)
    torch.cuda.synchronize()
    assert idv.status == 0 and idv.passes == 3
    assert np.linalg.norm(Rd.cpu().numpy() - Re) / np.linalg.norm(Re) <= 1e-12


def _timed_out_run(Xh, scope, fused=True):
    scqr3.debug_set(scqr3.DEBUG_WAIT_SCOPE, scope)
    scqr3.debug_set(scqr3.DEBUG_WAIT_NS, 0)
    try:
        return run(Xh, fused=fused)
    finally:
        scqr3.debug_set(scqr3.DEBUG_WAIT_NS, -1)
        scqr3.debug_set(scqr3.DEBUG_WAIT_SCOPE, 3)


@pytest.mark.parametrize("n,scope,fused", [(64, 1, True), (64, 2, True), (32, 2, True), (100, 1, True),
                                           (100, 2, True), (48, 2, False)])
def test_timeout_path_then_normal_call(n, scope, fused):
    """With the hand-off wait limit at zero for one kind of tensor-core kernel
    (scope 1: the Gram kernel; scope 2: the one-sweep substitution, or with
    fused=False / n > 64 the separate update kernel), that kernel's first wait
    that is not already satisfied gives up: the call reports SCQR3_E_TIMEOUT.
    The kernel still waits, with the normal limit, for its own MMAs and copies
    before it frees its tensor memory, so the next call on the same stream,
    with the default limit restored, returns the same bits as before."""
    Xh = testmat(200000, n, 1e8, seed=9800 + n + 10 * scope)
    Q0, R0, i0 = run(Xh, fused=fused)
    assert i0.status == 0
    _, _, it = _timed_out_run(Xh, scope, fused=fused)
    assert it.status == scqr3.E_TIMEOUT, (n, scope, it)
    Q1, R1, i1 = run(Xh, fused=fused)
    assert i1.status == 0 and i1.passes == i0.passes
    assert np.array_equal(Q1, Q0) and np.array_equal(R1, R0)
