"""Mixed form (FP32 pairs for the bulk, FP64 accumulation / shift / Cholesky)
against the FP64 CPU oracle.

Its unit roundoff is about 2^-48 instead of 2^-53, so R agrees with the FP64
oracle to about kappa * 2^-48 (relative) and the residual is O(2^-48); the
orthogonality target is the FP64 one, ||Q^T Q - I||_2 <= 1e-13, since the
Gram matrices are accumulated with FP64-level worst-case error.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1809_11085_gb300 import scqr3  # noqa: E402
from paper_1809_11085_gb300.testmat import repeated_small_sigma, testmat  # noqa: E402

pytestmark = pytest.mark.gpu
UDF = 2.0 ** -48


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1809_11085_gb300 import build

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run(Xh, **kw):
    X = torch.from_numpy(Xh).cuda()
    Q, R, info = scqr3.factor(X, precision=scqr3.PREC_MIXED, **kw)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), R.cpu().numpy(), info


def measures(Xh, Q, R, Ro):
    n = Q.shape[1]
    orth = np.linalg.norm(Q.T @ Q - np.eye(n), 2)
    res = np.linalg.norm(Xh - Q @ R) / np.linalg.norm(Xh)
    dR = np.linalg.norm(R - Ro) / np.linalg.norm(Ro)
    return orth, res, dR


@pytest.mark.parametrize("kappa", [1e4, 1e7, 1e10])
def test_mixed_config_shape_n128(kappa):
    m, n = 100000, 128
    Xh = testmat(m, n, kappa, seed=3000 + int(np.log10(kappa)))
    Q, R, info = run(Xh)
    assert info.status == 0, info
    _, Ro, st, tr = oracle.scqr3(Xh)
    assert st == 0
    orth, res, dR = measures(Xh, Q, R, Ro)
    assert orth <= 1e-13, orth
    assert res <= 64 * n * UDF, res
    assert dR <= max(1e-12, 100 * n * kappa * UDF), dR


@pytest.mark.parametrize("n", [1, 7, 16, 33, 64, 100, 128])
def test_mixed_shape_sweep(n):
    m = 4096 * 2 + 37
    Xh = testmat(m, n, 1e8, seed=3100 + n)
    Q, R, info = run(Xh)
    assert info.status == 0, info
    _, Ro, st, _ = oracle.scqr3(Xh)
    orth, res, dR = measures(Xh, Q, R, Ro)
    assert orth <= 1e-13 and res <= 64 * max(n, 8) * UDF, (orth, res)
    assert np.array_equal(np.tril(R, -1), np.zeros((n, n))) and (np.diag(R) > 0).all()


@pytest.mark.parametrize("kappa", [1e14, 1e15])
def test_mixed_extra_passes(kappa):
    m, n = 60000, 64
    Xh = testmat(m, n, kappa, seed=3200 + int(np.log10(kappa)))
    Q, R, info = run(Xh)
    assert info.status == 0, info
    assert info.shifted[0] == 1 and info.shifted[-2:] == [0, 0]
    n = Xh.shape[1]
    assert np.linalg.norm(Q.T @ Q - np.eye(n), 2) <= 1e-13


def test_mixed_repeated_sigma_and_in_place():
    m, n = 50000, 64
    Xh = testmat(m, n, 0.0, seed=3300, sigma=repeated_small_sigma(n, 8, 1e-14, 1e7))
    X = torch.from_numpy(Xh).cuda()
    Q, R, info = scqr3.factor(X, Q=X, precision=scqr3.PREC_MIXED)
    torch.cuda.synchronize()
    assert info.status == 0
    Qh = X.cpu().numpy()
    assert np.linalg.norm(Qh.T @ Qh - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(Xh - Qh @ R.cpu().numpy()) / np.linalg.norm(Xh) <= 64 * n * UDF


def test_mixed_matches_fp64_pass_sequence_far_from_threshold():
    Xh = testmat(30000, 32, 1e6, seed=3400)
    _, _, info = run(Xh)
    _, _, st, tr = oracle.scqr3(Xh)
    assert info.passes == tr["passes"] and info.shifted == tr["shifted"]


def test_mixed_rejects_oblique():
    X = torch.zeros((64, 8), dtype=torch.float64, device="cuda")
    B = torch.eye(8, dtype=torch.float64, device="cuda").repeat(8, 1, 1)
    with pytest.raises(scqr3.ScqrError):
        scqr3.factor(X, B, precision=scqr3.PREC_MIXED)
