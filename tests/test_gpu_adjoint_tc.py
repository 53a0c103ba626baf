"""The tensor-core adjoint (scqr3_backward_ex with SCQR3_PREC_TC, through the
C ABI) against the oracle's gradient references, against the FP64 adjoint,
and through autograd against central differences.

Tolerances are those of the FP64 adjoint (tests/test_gpu_adjoint.py): the
adjoint applies R_k^{-T} once per pass, so rounding differences are amplified
by about kappa_2(X); both forms are compared with the oracle within
50 n kappa u (relative, Frobenius). The shapes cover the one-sweep
substitution (16 < n <= 64), the separate-launch one (n <= 16, n > 64, and
16 < n <= 64 with the one-sweep form switched off), partial column blocks
(n not a multiple of 16 or 32) and ragged row tails.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.adjoint import passwise_adjoint, qr_adjoint  # noqa: E402
from paper_1809_11085_gb300 import batched, scqr3  # noqa: E402
from paper_1809_11085_gb300.testmat import testmat, testmat_torch  # noqa: E402

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
    scqr3.debug_set(scqr3.DEBUG_WAIT_SCOPE, 3)


def forward(Xh, precision=scqr3.PREC_FP64):
    X = torch.from_numpy(Xh).cuda()
    n = Xh.shape[1]
    Rpass = torch.zeros((scqr3.MAX_PASSES, n, n), dtype=torch.float64, device="cuda")
    Q, R, info = scqr3.factor(X, Rpass=Rpass, precision=precision)
    torch.cuda.synchronize()
    assert info.status == 0
    return Q, R, Rpass, info


def tc_backward(Q, Rpass, passes, dQ, dR, fused=True, **kw):
    m, n = Q.shape
    ws = scqr3.BackwardWorkspace(m, n, precision=TC)
    scqr3.debug_set(scqr3.DEBUG_FUSED_SOLVE, 1 if fused else 0)
    try:
        dX = scqr3.backward(Q, Rpass, passes, dQ, dR, workspace=ws, **kw)
        torch.cuda.synchronize()
    finally:
        scqr3.debug_set(scqr3.DEBUG_FUSED_SOLVE, 1)
    return dX, ws.last_status()


@pytest.mark.parametrize("n", [1, 3, 16, 20, 32, 48, 64, 65, 100, 128])
@pytest.mark.parametrize("kappa", [1e2, 1e6, 1e10])
def test_matches_oracle_references(n, kappa):
    m = 3000 + 7 * n
    rng = np.random.default_rng(1300 + n)
    Xh = testmat(m, n, kappa, seed=1400 + n)
    Q, R, Rpass, info = forward(Xh)
    dQh = rng.standard_normal((m, n))
    dRh = rng.standard_normal((n, n))
    dX, st = tc_backward(Q, Rpass, info.passes, torch.from_numpy(dQh).cuda(), torch.from_numpy(dRh).cuda())
    assert st == scqr3.OK
    g = dX.cpu().numpy()
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    tol = max(1e-12, 50 * n * kappa * U)
    ref = qr_adjoint(Qh, Rh, dQh, dRh)
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel < tol, (rel, tol)
    Rks = [Rpass[k].cpu().numpy() for k in range(info.passes)]
    ref2 = passwise_adjoint(Qh, Rks, dQh, dRh)
    rel2 = np.linalg.norm(g - ref2) / np.linalg.norm(ref2)
    assert rel2 < tol, (rel2, tol)


@pytest.mark.parametrize("n", [20, 48, 64])
def test_separate_launch_substitution(n):
    """16 < n <= 64 with the one-sweep substitution switched off: the same
    result as the one-sweep form within the oracle tolerance."""
    m = 5000 + 3 * n
    rng = np.random.default_rng(1500 + n)
    Xh = testmat(m, n, 1e6, seed=1600 + n)
    Q, R, Rpass, info = forward(Xh)
    dQ = torch.from_numpy(rng.standard_normal((m, n))).cuda()
    dR = torch.from_numpy(rng.standard_normal((n, n))).cuda()
    a, sa = tc_backward(Q, Rpass, info.passes, dQ, dR, fused=True)
    b, sb = tc_backward(Q, Rpass, info.passes, dQ, dR, fused=False)
    assert sa == sb == scqr3.OK
    ref = qr_adjoint(Q.cpu().numpy(), R.cpu().numpy(), dQ.cpu().numpy(), dR.cpu().numpy())
    tol = 50 * n * 1e6 * U
    for g in (a, b):
        assert np.linalg.norm(g.cpu().numpy() - ref) / np.linalg.norm(ref) < tol


@pytest.mark.parametrize("kappa,passes_min", [(1e14, 4), (1e15, 4)])
def test_extra_passes(kappa, passes_min):
    """Ill-conditioned X: the factorization took extra (shifted) passes and
    the adjoint walks back through all of them."""
    m, n = 6000, 32
    rng = np.random.default_rng(1700)
    Xh = testmat(m, n, kappa, seed=1701)
    Q, R, Rpass, info = forward(Xh)
    assert info.passes >= passes_min
    dQh = rng.standard_normal((m, n))
    dRh = rng.standard_normal((n, n))
    g, st = tc_backward(Q, Rpass, info.passes, torch.from_numpy(dQh).cuda(), torch.from_numpy(dRh).cuda())
    assert st == scqr3.OK
    fp = scqr3.backward(Q, Rpass, info.passes, torch.from_numpy(dQh).cuda(), torch.from_numpy(dRh).cuda())
    torch.cuda.synchronize()
    Rks = [Rpass[k].cpu().numpy() for k in range(info.passes)]
    ref = passwise_adjoint(Q.cpu().numpy(), Rks, dQh, dRh)
    tol = 50 * n * kappa * U
    for x in (g, fp):
        assert np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref) < tol


def test_after_the_tensor_core_forward():
    """Q and R_k from the SCQR3_PREC_TC factorization: the tensor-core and FP64
    adjoints of the same saved state agree, and both match the oracle."""
    m, n = 40000, 64
    rng = np.random.default_rng(1800)
    Xh = testmat(m, n, 1e8, seed=1801)
    Q, R, Rpass, info = forward(Xh, precision=TC)
    dQh = rng.standard_normal((m, n))
    dRh = rng.standard_normal((n, n))
    g, st = tc_backward(Q, Rpass, info.passes, torch.from_numpy(dQh).cuda(), torch.from_numpy(dRh).cuda())
    assert st == scqr3.OK
    fp = scqr3.backward(Q, Rpass, info.passes, torch.from_numpy(dQh).cuda(), torch.from_numpy(dRh).cuda())
    torch.cuda.synchronize()
    ref = qr_adjoint(Q.cpu().numpy(), R.cpu().numpy(), dQh, dRh)
    tol = 50 * n * 1e8 * U
    gn, fn = g.cpu().numpy(), fp.cpu().numpy()
    assert np.linalg.norm(gn - ref) / np.linalg.norm(ref) < tol
    assert np.linalg.norm(gn - fn) / np.linalg.norm(fn) < tol


def test_without_dR_and_in_place():
    m, n = 5000, 32
    Xh = testmat(m, n, 1e4, seed=1900)
    Q, R, Rpass, info = forward(Xh)
    dQ = torch.randn((m, n), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(19))
    ref = qr_adjoint(Q.cpu().numpy(), R.cpu().numpy(), dQ.cpu().numpy(), None)
    dX, st = tc_backward(Q, Rpass, info.passes, dQ, None, dX=dQ)  # in place over dQ
    assert st == scqr3.OK and dX.data_ptr() == dQ.data_ptr()
    g = dX.cpu().numpy()
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-11


def test_strided_inputs():
    """Q, dQ and dX as column slices of wider buffers (ld > n)."""
    m, n = 4000, 40
    rng = np.random.default_rng(2000)
    Xh = testmat(m, n, 1e5, seed=2001)
    Q, R, Rpass, info = forward(Xh)
    Qw = torch.zeros((m, n + 9), dtype=torch.float64, device="cuda")
    Qw[:, 3:3 + n] = Q
    dQh = rng.standard_normal((m, n))
    dQw = torch.zeros((m, n + 5), dtype=torch.float64, device="cuda")
    dQw[:, 1:1 + n] = torch.from_numpy(dQh).cuda()
    dXw = torch.full((m, n + 7), 7.0, dtype=torch.float64, device="cuda")
    ws = scqr3.BackwardWorkspace(m, n, precision=TC)
    scqr3.backward(Qw[:, 3:3 + n], Rpass, info.passes, dQw[:, 1:1 + n], None, dX=dXw[:, 2:2 + n], workspace=ws)
    torch.cuda.synchronize()
    assert ws.last_status() == scqr3.OK
    ref = qr_adjoint(Q.cpu().numpy(), R.cpu().numpy(), dQh, None)
    g = dXw[:, 2:2 + n].cpu().numpy()
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 50 * n * 1e5 * U
    assert torch.all(dXw[:, :2] == 7.0) and torch.all(dXw[:, 2 + n:] == 7.0)


def test_large_against_fp64_adjoint():
    """1,048,576 x 64 (the step's shape at 1/16 of the rows), kappa = 1e10:
    the tensor-core adjoint against the FP64 adjoint of the same saved state
    and against the oracle's closed form, whole dX."""
    m, n = 1 << 20, 64
    X, _, _ = testmat_torch(m, n, 1e10, seed=2100)
    Rpass = torch.zeros((scqr3.MAX_PASSES, n, n), dtype=torch.float64, device="cuda")
    Q, R, info = scqr3.factor(X, Rpass=Rpass, precision=TC)
    del X
    g = torch.Generator("cuda").manual_seed(21)
    dQ = torch.randn((m, n), dtype=torch.float64, device="cuda", generator=g)
    dR = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    a, st = tc_backward(Q, Rpass, info.passes, dQ, dR)
    assert st == scqr3.OK
    b = scqr3.backward(Q, Rpass, info.passes, dQ, dR)
    torch.cuda.synchronize()
    tol = 50 * n * 1e10 * U
    rel = (torch.linalg.matrix_norm(a - b) / torch.linalg.matrix_norm(b)).item()
    assert rel < tol, rel
    ref = qr_adjoint(Q.cpu().numpy(), R.cpu().numpy(), dQ.cpu().numpy(), dR.cpu().numpy())
    assert np.linalg.norm(a.cpu().numpy() - ref) / np.linalg.norm(ref) < tol


@pytest.mark.parametrize("n,fused", [(64, True), (100, False), (48, False)])
def test_timeout_path_then_normal_call(n, fused):
    """With the hand-off wait limit of the tensor-core substitution kernels at
    zero, the adjoint's status word reports SCQR3_E_TIMEOUT; the next call
    with the default limit gives the same bits as before."""
    m = 200000
    rng = np.random.default_rng(2200 + n)
    Xh = testmat(m, n, 1e6, seed=2201 + n)
    Q, R, Rpass, info = forward(Xh)
    dQ = torch.from_numpy(rng.standard_normal((m, n))).cuda()
    dR = torch.from_numpy(rng.standard_normal((n, n))).cuda()
    a, sa = tc_backward(Q, Rpass, info.passes, dQ, dR, fused=fused)
    assert sa == scqr3.OK
    scqr3.debug_set(scqr3.DEBUG_WAIT_SCOPE, 2)
    scqr3.debug_set(scqr3.DEBUG_WAIT_NS, 0)
    try:
        _, st = tc_backward(Q, Rpass, info.passes, dQ, dR, fused=fused)
    finally:
        scqr3.debug_set(scqr3.DEBUG_WAIT_NS, -1)
        scqr3.debug_set(scqr3.DEBUG_WAIT_SCOPE, 3)
    assert st == scqr3.E_TIMEOUT
    b, sb = tc_backward(Q, Rpass, info.passes, dQ, dR, fused=fused)
    assert sb == scqr3.OK
    assert torch.equal(a, b)


def test_repeatable():
    m, n = 30011, 56
    rng = np.random.default_rng(2300)
    Xh = testmat(m, n, 1e7, seed=2301)
    Q, R, Rpass, info = forward(Xh)
    dQ = torch.from_numpy(rng.standard_normal((m, n))).cuda()
    dR = torch.from_numpy(rng.standard_normal((n, n))).cuda()
    a, _ = tc_backward(Q, Rpass, info.passes, dQ, dR)
    b, _ = tc_backward(Q, Rpass, info.passes, dQ, dR)
    assert torch.equal(a, b)


@pytest.mark.parametrize("m,n,kappa", [(200, 16, 3e2), (500, 32, 1e3)])
def test_autograd_against_central_differences(m, n, kappa):
    """scqr3.qr with precision=PREC_TC (tensor-core forward and adjoint):
    loss = <W1, Q> + <W2, R> with seeded Gaussian W, h = 1e-6."""
    rng = np.random.default_rng(2400 + n)
    Xh = testmat(m, n, kappa, seed=2500 + n)
    W1 = torch.from_numpy(rng.standard_normal((m, n))).cuda()
    W2 = torch.from_numpy(rng.standard_normal((n, n))).cuda()

    def loss(X):
        Q, R = scqr3.qr(X, precision=TC)
        return (W1 * Q).sum() + (W2 * R).sum()

    X = torch.from_numpy(Xh).cuda().requires_grad_(True)
    (G,) = torch.autograd.grad(loss(X), X)
    h = 1e-6
    tol = 1e-6 + 10 * (h * kappa) ** 2 * kappa + 1e-9 * kappa
    with torch.no_grad():
        for t in range(3):
            D = torch.from_numpy(rng.standard_normal((m, n))).cuda()
            fd = (loss(X + h * D) - loss(X - h * D)).item() / (2 * h)
            an = (G * D).sum().item()
            assert abs(fd - an) <= tol * max(1.0, abs(an)), (t, fd, an, tol)


def test_gradcheck_tiny():
    X = torch.from_numpy(testmat(12, 3, 10.0, seed=2600)).cuda().requires_grad_(True)
    W = torch.randn(12, 3, dtype=torch.float64, device="cuda")

    def f(X):
        Q, R = scqr3.qr(X, precision=TC)
        return (W * Q).sum() + R.sum()

    assert torch.autograd.gradcheck(f, (X,), eps=1e-6, atol=1e-7, rtol=1e-6)


def test_batched_tensor_core_gradients():
    """qr_batched with PREC_TC: each matrix's gradient through the tensor-core
    adjoint against the closed-form adjoint of its own Q and R."""
    shapes = [(3000, 20), (5000, 64), (2500, 100), (700, 8)]
    rng = np.random.default_rng(2700)
    Xs = [torch.from_numpy(testmat(m, n, 1e6, seed=2701 + i)).cuda().requires_grad_(True)
          for i, (m, n) in enumerate(shapes)]
    Ws = [torch.from_numpy(rng.standard_normal((m, n))).cuda() for m, n in shapes]
    Vs = [torch.from_numpy(rng.standard_normal((n, n))).cuda() for _, n in shapes]
    Qs, Rs = batched.qr_batched(Xs, precision=TC)
    loss = sum((W * Q).sum() + (V * R).sum() for W, Q, V, R in zip(Ws, Qs, Vs, Rs))
    grads = torch.autograd.grad(loss, Xs)
    for (m, n), Q, R, W, V, g in zip(shapes, Qs, Rs, Ws, Vs, grads):
        ref = qr_adjoint(Q.detach().cpu().numpy(), R.detach().cpu().numpy(), W.cpu().numpy(), V.cpu().numpy())
        rel = np.linalg.norm(g.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert rel < 50 * n * 1e6 * U, (m, n, rel)


@pytest.mark.parametrize("kappa", [1e2, 1e10])
def test_full_size_sampled_rows_against_oracle(kappa):
    """16,777,216 x 64 (the bench's workload): the tensor-core forward and
    adjoint; 258 rows of dX (the first, the last and 256 seeded ones) against
    the oracle's closed form, with M = R dR^T - dQ^T Q summed on the host over
    1M-row chunks copied from the device."""
    from oracle.adjoint import qr_adjoint_rows

    m, n = 1 << 24, 64
    X, _, _ = testmat_torch(m, n, kappa, seed=2800)
    Rpass = torch.zeros((scqr3.MAX_PASSES, n, n), dtype=torch.float64, device="cuda")
    Q, R, info = scqr3.factor(X, Rpass=Rpass, precision=TC)
    del X
    assert info.status == 0
    g = torch.Generator("cuda").manual_seed(28)
    dQ = torch.randn((m, n), dtype=torch.float64, device="cuda", generator=g)
    dR = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    dX, st = tc_backward(Q, Rpass, info.passes, dQ, dR)
    assert st == scqr3.OK
    rows = np.concatenate([[0, m - 1], np.random.default_rng(29).choice(np.arange(1, m - 1), 256, replace=False)])
    ri = torch.from_numpy(rows).cuda()
    step = 1 << 20
    chunks = ((Q[a:a + step].cpu().numpy(), dQ[a:a + step].cpu().numpy()) for a in range(0, m, step))
    ref = qr_adjoint_rows(R.cpu().numpy(), dR.cpu().numpy(), chunks, Q[ri].cpu().numpy(), dQ[ri].cpu().numpy())
    got = dX[ri].cpu().numpy()
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < max(1e-12, 50 * n * kappa * U), rel
