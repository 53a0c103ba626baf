"""GPU parity of precision=SCQR3_PREC_TC: FP64 substitution with the Gram
matrices on the BF16 tensor cores through the exact seven-bit digit split
(n <= 128).

The split represents each entry to 2^-56 of its column's scale and every digit
product and 256-row sum is exact, so the Gram matrix is accurate to about
m 2^-55 sigma_j sigma_k: the same order as an FP64 Gram matrix. The tests
therefore use the FP64 parity tolerances against the oracle:
||Q^T Q - I||_2 <= 1e-13, ||X - QR||_F / ||X||_F <= 1e-13, and R within
1e-12 (kappa <= 1e8) or 100 n kappa u.
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


def run(Xh, **kw):
    Q, R, info = scqr3.factor(torch.from_numpy(Xh).cuda(), precision=TC, **kw)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), R.cpu().numpy(), info


def check(Xh, kappa, **kw):
    Qg, Rg, info = run(Xh, **kw)
    Qo, Ro, st, tr = oracle.scqr3(Xh, normx2=kw.get("norm_x2", 0.0), algorithm=kw.get("algorithm", 3))
    assert st == 0 and info.status == 0, (st, info)
    n = Xh.shape[1]
    assert np.array_equal(np.tril(Rg, -1), np.zeros((n, n)))
    assert (np.diag(Rg) > 0).all()
    assert np.linalg.norm(Qg.T @ Qg - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(Xh - Qg @ Rg) / np.linalg.norm(Xh) <= 1e-13
    dR = np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro)
    assert dR <= (1e-12 if kappa <= 1e8 else 100 * n * kappa * U), dR
    return info, tr


@pytest.mark.parametrize("n", [1, 2, 7, 16, 31, 32, 33, 63, 64, 65, 66, 96, 127, 128])
@pytest.mark.parametrize("m_kind", ["square", "small", "ragged", "tall"])
def test_shape_sweep(n, m_kind):
    """n <= 64: one 64-column block; 64 < n <= 128: the blocks (0,0), (1,1)
    and (0,1) on separate CTAs, 32-row chunks."""
    m = {"square": n, "small": 300, "ragged": 20011, "tall": 100003}[m_kind]
    if m < n:
        m = n
    Xh = testmat(m, n, 1e6, seed=6000 + n + m)
    check(Xh, 1e6)


@pytest.mark.parametrize("n", [129, 160, 192, 200, 255, 256])
@pytest.mark.parametrize("m_kind", ["square", "ragged", "tall"])
def test_wide_shape_sweep(n, m_kind):
    """128 < n <= 256: the Gram matrix as the ten 64-column block pairs (four
    diagonal, six off-diagonal) on separate CTA sets, the substitution in
    32-column diagonal blocks with the off-diagonal products on the tensor
    cores (up to 28 update launches per pass)."""
    m = {"square": n, "ragged": 20011, "tall": 60013}[m_kind]
    Xh = testmat(m, n, 1e6, seed=6300 + n + m)
    check(Xh, 1e6)


@pytest.mark.parametrize("kappa", [1e2, 1e10, 1e15])
def test_wide_conditioning(kappa):
    Xh = testmat(30011, 256, kappa, seed=6350)
    info, tr = check(Xh, kappa)
    if kappa <= 1e8:
        assert info.passes == tr["passes"]


def test_wide_matches_fp64_form():
    """n = 256 at 500,000 rows (each block pair's CTAs cover about 50 groups
    of 1024 rows): R within 1e-14 of the FP64 DFMA form, orthogonality and
    residual at the FP64 tolerances."""
    Xh = testmat(500000, 256, 1e8, seed=6360)
    X = torch.from_numpy(Xh).cuda()
    Qt, Rt, it = scqr3.factor(X, precision=TC)
    Qf, Rf, i_f = scqr3.factor(X)
    torch.cuda.synchronize()
    assert it.status == 0 and i_f.status == 0 and it.passes == i_f.passes
    Rt, Rf = Rt.cpu().numpy(), Rf.cpu().numpy()
    assert np.linalg.norm(Rt - Rf) / np.linalg.norm(Rf) <= 1e-14
    Qt = Qt.cpu().numpy()
    assert np.linalg.norm(Qt.T @ Qt - np.eye(256), 2) <= 1e-13
    assert np.linalg.norm(Xh - Qt @ Rt) / np.linalg.norm(Xh) <= 1e-13


def test_wide_host_form_and_shards():
    """n = 200 through the host-buffer entry point (row-chunked copies, the
    first Gram matrix per chunk) and through the row-partitioned calls
    (uneven blocks, Gram shares summed between the calls): both meet the FP64
    tolerances and match scqr3_factor's R to rounding."""
    m, n = 300000, 200
    Xh = testmat(m, n, 1e6, seed=6370)
    X = torch.from_numpy(Xh).cuda()
    Q1, R1, i1 = scqr3.factor(X, precision=TC)
    torch.cuda.synchronize()
    R1 = R1.cpu().numpy()
    Qh, Rh, ih = scqr3.factor_host(torch.from_numpy(Xh).pin_memory(), precision=TC)
    assert ih.status == 0 and ih.passes == i1.passes
    Qh, Rh = Qh.numpy(), Rh.numpy()
    assert np.linalg.norm(Qh.T @ Qh - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(Xh - Qh @ Rh) / np.linalg.norm(Xh) <= 1e-13
    assert np.linalg.norm(Rh - R1) / np.linalg.norm(R1) <= 1e-12
    bounds = [0, 70001, 70009, 210000, m]
    Xs = [X[a:b] for a, b in zip(bounds[:-1], bounds[1:])]
    wss = [scqr3.ShardWorkspace(b - a, n, None, 0.0, TC, 0) for a, b in zip(bounds[:-1], bounds[1:])]
    Qs = [torch.empty_like(x) for x in Xs]
    Rs = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in Xs]
    for x, ws in zip(Xs, wss):
        scqr3.gram_partial(x, ws, precision=TC)
    G = sum(ws.G for ws in wss)
    for k in range(6):
        for ws in wss:
            ws.G.copy_(G)
        for x, q, r, ws in zip(Xs, Qs, Rs, wss):
            scqr3.apply_pass(k, m, x, q, r, ws, precision=TC)
        torch.cuda.synchronize()
        inf = scqr3.Info.from_bytes(wss[0].info.cpu().numpy().tobytes())
        assert inf.status == 0
        if not inf.more:
            break
        G = sum(ws.G_next for ws in wss)
    Qs = torch.cat(Qs).cpu().numpy()
    Rs0 = Rs[0].cpu().numpy()
    for r in Rs[1:]:
        assert np.array_equal(r.cpu().numpy(), Rs0)
    assert np.linalg.norm(Qs.T @ Qs - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(Xh - Qs @ Rs0) / np.linalg.norm(Xh) <= 1e-13
    assert np.linalg.norm(Rs0 - R1) / np.linalg.norm(R1) <= 1e-12


@pytest.mark.parametrize("kappa", [1e2, 1e8, 1e12, 1e15])
def test_conditioning(kappa):
    """The pass structure follows the oracle's where the decisions are not
    marginal (kappa 1e2, 1e8: three passes; 1e15: a second shifted pass)."""
    Xh = testmat(50000, 64, kappa, seed=6100)
    info, tr = check(Xh, kappa, norm_x2=1.0)
    if kappa in (1e2, 1e8):
        assert info.passes == tr["passes"] == 3


@pytest.mark.parametrize("kappa", [1e2, 1e8, 1e15])
def test_conditioning_two_blocks(kappa):
    Xh = testmat(40000, 128, kappa, seed=6150)
    info, tr = check(Xh, kappa, norm_x2=1.0)
    if kappa in (1e2, 1e8):
        assert info.passes == tr["passes"] == 3


def test_block_grid_small_m():
    """m from 1 to a few read-back groups: CTAs of a block without rows still
    write their slot (zeros), and every block has at least one CTA."""
    for m, seed in ((100, 6160), (256, 6161), (257, 6162), (3 * 256 + 5, 6163), (40 * 256, 6164)):
        n = 100 if m >= 100 else m
        check(testmat(m, n, 1e5, seed=seed), 1e5)


@pytest.mark.parametrize("n,e", [(40, 300), (100, 200)])
def test_badly_scaled_columns_and_rows(n, e):
    """Column scales from 2^-e to 2^e and rows spanning 1e-30 .. 1: each
    column has its own power-of-two scale, and the fixed-point error is
    relative to it, which is what the norm-wise Gram bound needs. (The
    algorithm itself needs more passes as the column scales spread: the
    oracle takes 5 passes for the first case, 3 for the second, and 8 for
    n = 100 with e = 300.)"""
    rng = np.random.default_rng(6200 + n)
    m = 30000
    Xh = testmat(m, n, 1e4, seed=6201 + n)
    Xh *= np.exp2(rng.integers(-e, e, size=n))[None, :]
    Xh[rng.random(m) < 0.3] *= 1e-30
    Qg, Rg, info = run(Xh)
    assert info.status == 0
    Qd, Rd, idv = scqr3.factor(torch.from_numpy(Xh).cuda())
    Rd = Rd.cpu().numpy()
    assert info.passes == idv.passes
    # column scaling commutes with QR: compare R column-scaled
    scale = np.abs(np.diag(Rd))
    assert np.linalg.norm((Rg - Rd) / scale[None, :]) < 1e-10
    assert np.linalg.norm(Qg.T @ Qg - np.eye(n), 2) < 1e-13


@pytest.mark.parametrize("n", [64, 128])
def test_matches_fp64_form_at_scale(n):
    m = 1_000_000
    from paper_1809_11085_gb300.testmat import testmat_torch

    X, _, _ = testmat_torch(m, n, 1e8, seed=6300)
    Qt, Rt, it = scqr3.factor(X, precision=TC)
    Qd, Rd, idv = scqr3.factor(X)
    torch.cuda.synchronize()
    assert it.status == 0 and it.passes == idv.passes
    assert (torch.linalg.matrix_norm(Rt - Rd) / torch.linalg.matrix_norm(Rd)).item() < 1e-12
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    assert torch.linalg.matrix_norm(Qt.T @ Qt - eye, 2).item() < 1e-13
    assert (torch.linalg.matrix_norm(X - Qt @ Rt) / torch.linalg.matrix_norm(X)).item() < 1e-13


def test_deterministic_host_form_and_alg2():
    Xh = testmat(200000, 64, 1e10, seed=6400)
    Q1, R1, i1 = run(Xh)
    Q2, R2, i2 = run(Xh)
    assert np.array_equal(Q1, Q2) and np.array_equal(R1, R2)
    X = torch.empty(Xh.shape, dtype=torch.float64, pin_memory=True)
    X.copy_(torch.from_numpy(Xh))
    Qh, Rh, ih = scqr3.factor_host(X, precision=TC)  # one chunk: the same launches
    assert ih.status == 0
    assert np.array_equal(Qh.numpy(), Q1) and np.array_equal(Rh.numpy(), R1)
    check(testmat(100000, 48, 1e5, seed=6401), 1e5, algorithm=scqr3.ALG_ADAPTIVE)


def test_non_finite_and_rejections():
    Xh = testmat(5000, 16, 1e4, seed=6500)
    Xh[77, 3] = np.inf
    _, _, info = run(Xh)
    assert info.status == scqr3.E_NONFINITE
    with pytest.raises(scqr3.ScqrError):
        scqr3.factor(torch.zeros((1000, 257), dtype=torch.float64, device="cuda"), precision=TC)
    with pytest.raises(scqr3.ScqrError):
        scqr3.factor(torch.zeros((1000, 129), dtype=torch.float64, device="cuda"), precision=scqr3.PREC_MIXED_TC)
    Xh = testmat(5000, 100, 1e4, seed=6501)
    Xh[4321, 99] = np.nan  # a column of the second block
    _, _, info = run(Xh)
    assert info.status == scqr3.E_NONFINITE


# ------------------------------------------------------------------------------- mixed substitution + TC Gram

UDF = 2.0 ** -48


@pytest.mark.parametrize("n", [1, 7, 16, 33, 64, 65, 128])
@pytest.mark.parametrize("kappa", [1e4, 1e10, 1e15])
def test_mixed_tc_against_oracle(n, kappa):
    """PREC_MIXED_TC: the mixed form's FP32-pair substitution (unit roundoff
    about 2^-48) with the tensor-core Gram matrices; the tolerances are the
    mixed form's (orthogonality 1e-13, residual 64 n 2^-48, R to 100 n kappa 2^-48)."""
    m = 30011
    Xh = testmat(m, n, kappa, seed=6600 + n + int(np.log10(kappa)))
    Q, R, info = scqr3.factor(torch.from_numpy(Xh).cuda(), precision=scqr3.PREC_MIXED_TC)
    torch.cuda.synchronize()
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    _, Ro, st, tr = oracle.scqr3(Xh)
    assert st == 0 and info.status == 0, info
    assert np.linalg.norm(Q.T @ Q - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(Xh - Q @ R) / np.linalg.norm(Xh) <= 64 * max(n, 8) * UDF
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= max(1e-12, 100 * n * kappa * UDF)
    assert np.array_equal(np.tril(R, -1), np.zeros((n, n))) and (np.diag(R) > 0).all()


def test_mixed_tc_alg2_host_and_scale():
    from paper_1809_11085_gb300.testmat import testmat_torch

    X, _, _ = testmat_torch(1_000_000, 64, 1e10, seed=6700)
    Q, R, info = scqr3.factor(X, precision=scqr3.PREC_MIXED_TC)
    Qd, Rd, _ = scqr3.factor(X)
    torch.cuda.synchronize()
    assert info.status == 0 and info.passes == 3
    eye = torch.eye(64, dtype=torch.float64, device="cuda")
    assert torch.linalg.matrix_norm(Q.T @ Q - eye, 2).item() < 1e-13
    assert (torch.linalg.matrix_norm(X - Q @ R) / torch.linalg.matrix_norm(X)).item() < 64 * 64 * UDF
    Xh = testmat(100000, 48, 1e5, seed=6701)
    Qa, Ra, ia = scqr3.factor(torch.from_numpy(Xh).cuda(), precision=scqr3.PREC_MIXED_TC,
                              algorithm=scqr3.ALG_ADAPTIVE)
    torch.cuda.synchronize()
    assert ia.status == 0 and ia.passes == 2
    Xp = torch.empty(Xh.shape, dtype=torch.float64, pin_memory=True)
    Xp.copy_(torch.from_numpy(Xh))
    Qh, Rh, ih = scqr3.factor_host(Xp, precision=scqr3.PREC_MIXED_TC, algorithm=scqr3.ALG_ADAPTIVE)
    assert ih.status == 0
    assert np.array_equal(Qh.numpy(), Qa.cpu().numpy()) and np.array_equal(Rh.numpy(), Ra.cpu().numpy())


# ------------------------------------------------------------------ blocked substitution layouts

@pytest.mark.parametrize("n", [24, 40, 100, 128])
def test_in_place_leading_dimension_and_separate_output(n):
    """The substitution reads block 0 from the pass's input and updates and
    solves every later 32-column block in the output: in place (Q = X) with a
    leading dimension above n, and a separate Q with its own leading
    dimension, give the same bits, and the columns around the view stay
    untouched."""
    m = 20011
    Xh = testmat(m, n, 1e9, seed=6800 + n)
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
    assert torch.all(wide[:, :2] == 0) and torch.all(wide[:, 2 + n:] == 0)
    assert torch.all(outw[:, :1] == 7.0) and torch.all(outw[:, 1 + n:] == 7.0)
    Q, R = Qb.cpu().numpy(), Rb.cpu().numpy()
    assert np.linalg.norm(Q.T @ Q - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(Xh - Q @ R) / np.linalg.norm(Xh) <= 1e-13


@pytest.mark.parametrize("n", [100, 128])
def test_host_form_alg2_and_small_shift_wide(n):
    """factor_host runs the last substitution in row chunks (each one the full
    block sequence). With one chunk (m <= 262144) it makes the device call's
    launches and is bitwise equal to it; with three, the first Gram is summed
    per chunk, so the result differs at the rounding level amplified by kappa
    and is held to the FP64 tolerances instead. Alg. 2 and the smaller first
    shift go through the same blocked substitution."""
    for m, seed in ((200000, 6900 + n), (600000, 6950 + n)):
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
    check(testmat(60000, n, 1e5, seed=6910 + n), 1e5, algorithm=scqr3.ALG_ADAPTIVE)
    Qs, Rs, isv = run(testmat(60000, n, 1e7, seed=6920 + n), shift_scale=500.0)
    assert isv.status == 0
    assert np.linalg.norm(Qs.T @ Qs - np.eye(n), 2) <= 1e-13


# ------------------------------------------------------------------ oblique inner product (block-diagonal B)

def orth_b(Q, Bblk):
    n, bs = Q.shape[1], Bblk.shape[1]
    BQ = np.einsum("kij,kjn->kin", Bblk, Q.reshape(-1, bs, n)).reshape(Q.shape)
    return np.linalg.norm(Q.T @ BQ - np.eye(n), 2)


@pytest.mark.parametrize("n,bs,kappa,m", [(16, 8, 1e8, 24000), (40, 4, 1e10, 24004), (64, 8, 1e10, 24000),
                                          (100, 2, 1e6, 24002), (128, 8, 1e10, 24000), (33, 1, 1e4, 24001)])
def test_oblique_against_oracle(n, bs, kappa, m):
    """The Gram matrix of Z = L^T Q on the tensor cores (L_j^T applied to each
    8-row unit before the digit cut, the column scales from the same Z), with
    ||Q||_F^2 from the diagonal-block CTAs for the oblique shift, and the
    blocked substitution: B-orthogonality, residual and R against the oracle at
    the FP64 tolerances. m not a multiple of 8 leaves a last unit with fewer
    rows than 8 (whole blocks of bs rows)."""
    from paper_1809_11085_gb300.testmat import block_diag_spd

    Xh = testmat(m, n, kappa, seed=7000 + n + bs)
    Bh = block_diag_spd(m, bs, seed=7100 + n + bs)
    Q, R, info = scqr3.factor(torch.from_numpy(Xh).cuda(), torch.from_numpy(Bh).cuda(), precision=TC)
    torch.cuda.synchronize()
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    Qo, Ro, st, tr = oracle.scqr3(Xh, Bblk=Bh)
    assert st == 0 and info.status == 0, info
    assert info.passes == tr["passes"]
    assert orth_b(Q, Bh) <= 1e-13
    assert np.linalg.norm(Xh - Q @ R) / np.linalg.norm(Xh) <= 1e-13
    dR = np.linalg.norm(R - Ro) / np.linalg.norm(Ro)
    assert dR <= (1e-12 if kappa <= 1e8 else 100 * n * kappa * U), dR


def test_oblique_matches_fp64_form_and_host_and_rejections():
    """At kappa 1e8 the pass decisions are clear and the tensor-core form
    takes the FP64 form's passes; at kappa 1e10 (with kappa(B) ~ 1e3) the
    plain Cholesky of the second pass sits at the margin (kappa(Q_1)^2 u near
    1), where either form may add the breakdown rule's shifted pass, so only
    the results are compared there."""
    from paper_1809_11085_gb300.testmat import block_diag_spd

    m, n = 400000, 64
    Bb = torch.from_numpy(block_diag_spd(m, 8, seed=7201)).cuda()
    Bh = Bb.cpu().numpy()
    for kappa, seed in ((1e8, 7200), (1e10, 7202)):
        Xh = testmat(m, n, kappa, seed=seed)
        X = torch.from_numpy(Xh).cuda()
        Qt, Rt, it = scqr3.factor(X, Bb, precision=TC)
        Qd, Rd, idv = scqr3.factor(X, Bb)
        torch.cuda.synchronize()
        assert it.status == 0 and idv.status == 0
        if kappa <= 1e8:
            assert it.passes == idv.passes
            assert (torch.linalg.matrix_norm(Rt - Rd) / torch.linalg.matrix_norm(Rd)).item() < 1e-12
        assert orth_b(Qt.cpu().numpy(), Bh) <= 1e-13
        assert (torch.linalg.matrix_norm(X - Qt @ Rt) / torch.linalg.matrix_norm(X)).item() <= 1e-13
    Xp = torch.empty(Xh.shape, dtype=torch.float64, pin_memory=True)
    Xp.copy_(torch.from_numpy(Xh))
    Qh, Rh, ih = scqr3.factor_host(Xp, Bb, precision=TC)
    assert ih.status == 0
    assert orth_b(Qh.numpy(), Bh) <= 1e-13
    # blocks of 16 rows and a CSR B stay on FP64; the mixed substitution takes no B
    with pytest.raises(scqr3.ScqrError):
        scqr3.factor(X[:64000], torch.from_numpy(block_diag_spd(64000, 16, seed=1)).cuda(), precision=TC)
    with pytest.raises(scqr3.ScqrError):
        scqr3.factor(X[:64000], Bb[:8000], precision=scqr3.PREC_MIXED_TC)
