"""Batched form: every matrix of a batch against the single-matrix call and
the CPU oracle; determinism under CUDA-graph replay and re-runs; tile-shape
changes; gradients of the differentiable batch against central differences.

The batched partial Gram sums are grouped by tile instead of by CTA, so
results equal the single-matrix call to rounding (not bit for bit); they are
bitwise reproducible across runs and graph replays of one plan.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1809_11085_gb300 import batched, scqr3  # noqa: E402
from paper_1809_11085_gb300.testmat import batched_shapes, testmat  # noqa: E402

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1809_11085_gb300 import build

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def mixed_batch(seed=5000):
    rng = np.random.default_rng(seed)
    shapes = [(300, 1), (301, 5), (2000, 16), (777, 17), (5000, 32), (4097, 31), (6000, 48),
              (9000, 64), (257, 64), (3000, 100), (12000, 128), (129, 128), (20000, 16), (15000, 64)]
    mats = []
    for i, (m, n) in enumerate(shapes):
        kappa = 10 ** rng.uniform(2, 12)
        mats.append((testmat(m, n, kappa, seed=seed + i), kappa))
    return mats


def orth2(Q):
    n = Q.shape[1]
    return np.linalg.norm(Q.T @ Q - np.eye(n), 2)


def test_batch_matches_single_calls_and_oracle():
    mats = mixed_batch()
    Xs = [torch.from_numpy(x).cuda() for x, _ in mats]
    b = batched.BatchedQR(Xs)
    b.run()
    torch.cuda.synchronize()
    infos = b.infos()
    for i, ((xh, kappa), Q, R, inf) in enumerate(zip(mats, b.Qs, b.Rs, infos)):
        assert inf.status == 0, (i, inf)
        Qg, Rg = Q.cpu().numpy(), R.cpu().numpy()
        n = xh.shape[1]
        assert orth2(Qg) <= 1e-13, i
        assert np.linalg.norm(xh - Qg @ Rg) / np.linalg.norm(xh) <= 1e-13, i
        assert np.array_equal(np.tril(Rg, -1), np.zeros((n, n))) and (np.diag(Rg) > 0).all()
        Qs, Rs, infs = scqr3.factor(torch.from_numpy(xh).cuda())
        Rs = Rs.cpu().numpy()
        _, Ro, st, tr = oracle.scqr3(xh)
        tol = max(1e-12, 100 * n * kappa * U)
        assert np.linalg.norm(Rg - Rs) / np.linalg.norm(Rs) <= tol, i
        assert np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro) <= tol, i


def test_graph_replay_and_reruns_are_bitwise_identical():
    mats = mixed_batch(5100)
    Xs = [torch.from_numpy(x).cuda() for x, _ in mats]
    eager = batched.BatchedQR(Xs)
    eager.run()
    torch.cuda.synchronize()
    ref = [(q.clone(), r.clone()) for q, r in zip(eager.Qs, eager.Rs)]
    eager.run()
    torch.cuda.synchronize()
    for (q, r), q2, r2 in zip(ref, eager.Qs, eager.Rs):
        assert torch.equal(q, q2) and torch.equal(r, r2)
    g = batched.BatchedQR(Xs, graph=True)
    for _ in range(2):
        for Q in g.Qs:
            Q.fill_(float("nan"))
        g.run()
        torch.cuda.synchronize()
        for (q, r), q2, r2 in zip(ref, g.Qs, g.Rs):
            assert torch.equal(q, q2) and torch.equal(r, r2)
    assert all(i.status == 0 for i in g.infos())


@pytest.mark.parametrize("tp", [1, 3, 32])
def test_tile_shapes_agree(tp):
    mats = mixed_batch(5200)
    Xs = [torch.from_numpy(x).cuda() for x, _ in mats]
    a = batched.BatchedQR(Xs, tune=batched.tuning(8))
    b = batched.BatchedQR(Xs, tune=batched.tuning(tp))
    a.run()
    b.run()
    torch.cuda.synchronize()
    for (xh, kappa), Ra, Rb in zip(mats, a.Rs, b.Rs):
        n = xh.shape[1]
        d = (torch.linalg.matrix_norm(Ra - Rb) / torch.linalg.matrix_norm(Ra)).item()
        assert d <= max(1e-12, 100 * n * kappa * U)


def test_in_place_batch():
    mats = mixed_batch(5300)
    Xs = [torch.from_numpy(x).cuda() for x, _ in mats]
    b = batched.BatchedQR(Xs, in_place=True)
    b.run()
    torch.cuda.synchronize()
    for (xh, _), X, R in zip(mats, Xs, b.Rs):
        Qg = X.cpu().numpy()
        assert orth2(Qg) <= 1e-13
        assert np.linalg.norm(xh - Qg @ R.cpu().numpy()) / np.linalg.norm(xh) <= 1e-13


def test_config_mix_small_m():
    """The batched config's mix of n and kappa (512 matrices), with m shrunk to keep the test short."""
    shapes = batched_shapes(512, seed=77, m_lo=200, m_hi=3000)
    Xs = [torch.from_numpy(testmat(m, n, k, seed=6000 + i)).cuda() for i, (m, n, k) in enumerate(shapes)]
    b = batched.BatchedQR(Xs, graph=True)
    b.run()
    torch.cuda.synchronize()
    infos = b.infos()
    assert all(i.status == 0 for i in infos)
    worst = 0.0
    for X, Q, R in zip(Xs, b.Qs, b.Rs):
        n = X.shape[1]
        G = Q.T @ Q - torch.eye(n, dtype=torch.float64, device="cuda")
        worst = max(worst, torch.linalg.matrix_norm(G, 2).item())
        res = (torch.linalg.matrix_norm(X - Q @ R) / torch.linalg.matrix_norm(X)).item()
        assert res <= 1e-13
    assert worst <= 1e-13


def test_differentiable_batch_against_central_differences():
    """loss = sum_i <W1_i, Q_i> + <W2_i, R_i> on 8 matrices with m <= 500, h = 1e-6."""
    rng = np.random.default_rng(7000)
    shapes = [(120, 16), (200, 32), (480, 64), (500, 16), (333, 32), (260, 128), (450, 64), (150, 17)]
    kappas = [10 ** rng.uniform(2, 3) for _ in shapes]
    Xh = [testmat(m, n, k, seed=7100 + i) for i, ((m, n), k) in enumerate(zip(shapes, kappas))]
    W1 = [torch.from_numpy(rng.standard_normal(x.shape)).cuda() for x in Xh]
    W2 = [torch.from_numpy(rng.standard_normal((x.shape[1], x.shape[1]))).cuda() for x in Xh]

    def loss(Xs):
        Qs, Rs = batched.qr_batched(Xs)
        return sum((a * q).sum() + (b * r).sum() for a, b, q, r in zip(W1, W2, Qs, Rs))

    Xs = [torch.from_numpy(x).cuda().requires_grad_(True) for x in Xh]
    L = loss(Xs)
    grads = torch.autograd.grad(L, Xs)
    # each gradient against the oracle's closed-form QR adjoint of the computed factors
    from oracle.adjoint import qr_adjoint
    with torch.no_grad():
        Qs, Rs = batched.qr_batched([x.detach() for x in Xs])
    for i, (g, q, r) in enumerate(zip(grads, Qs, Rs)):
        ref = qr_adjoint(q.cpu().numpy(), r.cpu().numpy(), W1[i].cpu().numpy(), W2[i].cpu().numpy())
        rel = np.linalg.norm(g.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert rel < max(1e-12, 50 * q.shape[1] * kappas[i] * U), (i, rel)
    # central differences: truncation error ~ (h kappa)^2 kappa, plus u/h
    h = 1e-6
    kmax = max(kappas)
    tol = 1e-6 + 10 * (h * kmax) ** 2 * kmax
    with torch.no_grad():
        for t in range(3):
            D = [torch.from_numpy(rng.standard_normal(x.shape)).cuda() for x in Xh]
            fd = (loss([x + h * d for x, d in zip(Xs, D)]) - loss([x - h * d for x, d in zip(Xs, D)])).item() / (2 * h)
            an = sum((g * d).sum().item() for g, d in zip(grads, D))
            assert abs(fd - an) <= tol * max(1.0, abs(an)), (t, fd, an, tol)


def test_batch_options_alg2_and_small_shift():
    """shift_scale, algorithm and tol reach every matrix of a batch (Alg. 2's
    default tolerance from each matrix's own m, n): the pass counts of the
    single calls with the same options, and their results to rounding. The
    condition numbers keep Alg. 2's stopping test away from its margin: one
    plain pass leaves ||Q^T Q - I|| ~ kappa^2 u, at least 16 times the
    tolerance 6 (mn + n(n+1)) u here, so CholeskyQR2 (two passes) stops it."""
    shapes = [(3000, 16, 1e4), (5000, 32, 1e5), (9000, 64, 1e4), (4000, 100, 1e5), (7000, 128, 1e4)]
    mats = [testmat(m, n, k, seed=5900 + i) for i, (m, n, k) in enumerate(shapes)]
    for opts in ({"algorithm": scqr3.ALG_ADAPTIVE}, {"shift_scale": 500.0}):
        Xs = [torch.from_numpy(x).cuda() for x in mats]
        b = batched.BatchedQR(Xs, **opts)
        b.run()
        torch.cuda.synchronize()
        for i, (xh, inf, Q, R) in enumerate(zip(mats, b.infos(), b.Qs, b.Rs)):
            Qs, Rs, isg = scqr3.factor(torch.from_numpy(xh).cuda(), **opts)
            torch.cuda.synchronize()
            assert inf.status == 0 and isg.status == 0, (i, inf, isg)
            assert inf.passes == isg.passes, (opts, i, inf.passes, isg.passes)
            if "algorithm" in opts:
                assert inf.passes == 2
            Rg, Rsn = R.cpu().numpy(), Rs.cpu().numpy()
            assert np.linalg.norm(Rg - Rsn) / np.linalg.norm(Rsn) <= 1e-12
            m, n = xh.shape
            tol = 6 * (m * n + n * (n + 1)) * U if "algorithm" in opts else 1e-13
            assert orth2(Q.cpu().numpy()) <= tol


@pytest.mark.parametrize("prec", [scqr3.PREC_TC, scqr3.PREC_MIXED_TC])
def test_tensor_core_batch_graph(prec):
    """precision = PREC_TC / PREC_MIXED_TC: one scqr3_factor call per matrix on
    one shared workspace, captured as one CUDA graph. Each matrix equals the
    single call of that precision bit for bit (the same kernels and sums; the
    shared workspace is larger than a single shape needs, which changes no
    layout), every replay reproduces it, and every matrix meets the FP64
    tolerances against the oracle (the mixed form its own, looser residual)."""
    mats = mixed_batch(5600) + [(testmat(6000, 200, 1e8, seed=5650), 1e8)] if prec == scqr3.PREC_TC \
        else mixed_batch(5600)
    Xs = [torch.from_numpy(x).cuda() for x, _ in mats]
    g = batched.BatchedQR(Xs, graph=True, precision=prec)
    for rep in range(2):
        for Q in g.Qs:
            Q.fill_(float("nan"))
        g.run()
        torch.cuda.synchronize()
        infos = g.infos()
        for (xh, kappa), X, Qb, Rb, inf in zip(mats, Xs, g.Qs, g.Rs, infos):
            assert inf.status == 0
            Q1, R1, i1 = scqr3.factor(X, precision=prec)
            torch.cuda.synchronize()
            assert i1.passes == inf.passes
            assert torch.equal(Qb, Q1) and torch.equal(Rb, R1)
            if rep == 0:
                n = xh.shape[1]
                Qh, Rh = Qb.cpu().numpy(), Rb.cpu().numpy()
                _, Ro, st, _ = oracle.scqr3(xh)
                assert st == 0
                assert orth2(Qh) <= 1e-13
                res = np.linalg.norm(xh - Qh @ Rh) / np.linalg.norm(xh)
                assert res <= (1e-13 if prec == scqr3.PREC_TC else 64 * n * 2.0 ** -48)
                tol = max(1e-12, 100 * n * kappa * (U if prec == scqr3.PREC_TC else 2.0 ** -48))
                assert np.linalg.norm(Rh - Ro) / np.linalg.norm(Ro) <= tol


def test_differentiable_tensor_core_batch():
    """qr_batched(precision=PREC_TC): the forward pass through the tensor-core
    batch (one graph-capturable sequence of per-matrix calls), the backward
    through the adjoint with one shared workspace; every gradient against the
    oracle's closed-form QR adjoint of the computed factors."""
    rng = np.random.default_rng(7300)
    shapes = [(3000, 16), (2000, 32), (4800, 64), (500, 16), (3333, 48), (2600, 128), (150, 17)]
    kappas = [10 ** rng.uniform(2, 6) for _ in shapes]
    Xh = [testmat(m, n, k, seed=7400 + i) for i, ((m, n), k) in enumerate(zip(shapes, kappas))]
    W1 = [torch.from_numpy(rng.standard_normal(x.shape)).cuda() for x in Xh]
    W2 = [torch.from_numpy(rng.standard_normal((x.shape[1], x.shape[1]))).cuda() for x in Xh]
    Xs = [torch.from_numpy(x).cuda().requires_grad_(True) for x in Xh]
    Qs, Rs = batched.qr_batched(Xs, precision=scqr3.PREC_TC)
    L = sum((a * q).sum() + (b * r).sum() for a, b, q, r in zip(W1, W2, Qs, Rs))
    grads = torch.autograd.grad(L, Xs)
    from oracle.adjoint import qr_adjoint
    for i, (g, q, r) in enumerate(zip(grads, Qs, Rs)):
        q, r = q.detach().cpu().numpy(), r.detach().cpu().numpy()
        assert orth2(q) <= 1e-13
        ref = qr_adjoint(q, r, W1[i].cpu().numpy(), W2[i].cpu().numpy())
        rel = np.linalg.norm(g.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert rel < max(1e-12, 50 * q.shape[1] * kappas[i] * U), (i, rel)
