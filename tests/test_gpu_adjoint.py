"""GPU adjoint (scqr3_backward through the C ABI) against the oracle's
gradient references and against central finite differences.

Tolerances: the adjoint applies R_k^{-T} once per pass, so rounding
differences are amplified by about kappa_2(X); we compare to the oracle
within 50 n kappa u (relative, Frobenius). Central differences with
h = 1e-6 carry a truncation error of order h^2 kappa^3 (plus u/h), so they
are checked on small, well-conditioned matrices (kappa <= 1e3, m <= 500).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle.adjoint import passwise_adjoint, qr_adjoint  # noqa: E402
from paper_1809_11085_gb300 import scqr3  # noqa: E402
from paper_1809_11085_gb300.testmat import testmat  # noqa: E402

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1809_11085_gb300 import build

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def gpu_forward(Xh):
    X = torch.from_numpy(Xh).cuda()
    n = Xh.shape[1]
    Rpass = torch.zeros((scqr3.MAX_PASSES, n, n), dtype=torch.float64, device="cuda")
    Q, R, info = scqr3.factor(X, Rpass=Rpass)
    torch.cuda.synchronize()
    assert info.status == 0
    return Q, R, Rpass, info


@pytest.mark.parametrize("n", [3, 16, 32, 64, 100, 128])
@pytest.mark.parametrize("kappa", [1e2, 1e6, 1e10])
def test_backward_matches_oracle_references(n, kappa):
    m = 3000 + 7 * n
    rng = np.random.default_rng(300 + n)
    Xh = testmat(m, n, kappa, seed=400 + n)
    Q, R, Rpass, info = gpu_forward(Xh)
    dQh = rng.standard_normal((m, n))
    dRh = rng.standard_normal((n, n))
    dX = scqr3.backward(Q, Rpass, info.passes, torch.from_numpy(dQh).cuda(),
                        torch.from_numpy(dRh).cuda())
    torch.cuda.synchronize()
    g = dX.cpu().numpy()
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    ref = qr_adjoint(Qh, Rh, dQh, dRh)
    tol = max(1e-12, 50 * n * kappa * U)
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel < tol, (rel, tol)
    Rks = [Rpass[k].cpu().numpy() for k in range(info.passes)]
    ref2 = passwise_adjoint(Qh, Rks, dQh, dRh)
    rel2 = np.linalg.norm(g - ref2) / np.linalg.norm(ref2)
    assert rel2 < tol, (rel2, tol)


def test_backward_without_dR_and_in_place():
    m, n = 5000, 32
    Xh = testmat(m, n, 1e4, seed=500)
    Q, R, Rpass, info = gpu_forward(Xh)
    dQ = torch.randn((m, n), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    ref = qr_adjoint(Q.cpu().numpy(), R.cpu().numpy(), dQ.cpu().numpy(), None)
    dX = scqr3.backward(Q, Rpass, info.passes, dQ, None, dX=dQ)  # in place over dQ
    torch.cuda.synchronize()
    assert dX.data_ptr() == dQ.data_ptr()
    g = dX.cpu().numpy()
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-11


@pytest.mark.parametrize("m,n,kappa", [(60, 4, 1e2), (200, 16, 3e2), (500, 32, 1e3)])
def test_autograd_against_central_differences(m, n, kappa):
    """loss = <W1, Q> + <W2, R> with seeded Gaussian W, h = 1e-6."""
    rng = np.random.default_rng(600 + n)
    Xh = testmat(m, n, kappa, seed=700 + n)
    W1 = torch.from_numpy(rng.standard_normal((m, n))).cuda()
    W2 = torch.from_numpy(rng.standard_normal((n, n))).cuda()

    def loss(X):
        Q, R = scqr3.qr(X)
        return (W1 * Q).sum() + (W2 * R).sum()

    X = torch.from_numpy(Xh).cuda().requires_grad_(True)
    L = loss(X)
    (G,) = torch.autograd.grad(L, X)
    h = 1e-6
    tol = 1e-6 + 10 * (h * kappa) ** 2 * kappa + 1e-9 * kappa
    with torch.no_grad():
        for t in range(3):
            D = torch.from_numpy(rng.standard_normal((m, n))).cuda()
            fd = (loss(X + h * D) - loss(X - h * D)).item() / (2 * h)
            an = (G * D).sum().item()
            assert abs(fd - an) <= tol * max(1.0, abs(an)), (t, fd, an, tol)


def test_gradcheck_tiny():
    X = torch.from_numpy(testmat(12, 3, 10.0, seed=800)).cuda().requires_grad_(True)
    W = torch.randn(12, 3, dtype=torch.float64, device="cuda")

    def f(X):
        Q, R = scqr3.qr(X)
        return (W * Q).sum() + R.sum()

    assert torch.autograd.gradcheck(f, (X,), eps=1e-6, atol=1e-7, rtol=1e-6)
