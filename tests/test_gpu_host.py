"""scqr3_factor_host (X, Q, R, info in host memory) against scqr3_factor.

Up to 262,144 rows the host form makes the same launches as scqr3_factor
(one chunk), so the results are bit for bit equal; with B != I the first
Gram matrix is never split, so they are equal at any size. Above that, with
B = I, each row chunk of X writes its own partial Gram sums as it arrives, so
the first Gram matrix is summed in another order: R then agrees to the FP64
parity tolerance (1e-12 for kappa <= 1e8) and Q to its orthogonality bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1809_11085_gb300 import scqr3  # noqa: E402
from paper_1809_11085_gb300.testmat import block_diag_spd, laplacian_csr, testmat  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1809_11085_gb300 import build

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def pinned(a):
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    t.copy_(torch.from_numpy(a))
    return t


def device_run(Xh, B=None, **kw):
    Q, R, info = scqr3.factor(torch.from_numpy(Xh).cuda(), B, **kw)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), R.cpu().numpy(), info


@pytest.mark.parametrize("n", [7, 16, 64, 128, 200])
@pytest.mark.parametrize("kappa", [1e4, 1e14])
def test_single_chunk_is_bitwise_equal(n, kappa):
    Xh = testmat(60000 + n, n, kappa, seed=5000 + n)
    Qd, Rd, idv = device_run(Xh)
    Q, R, info = scqr3.factor_host(pinned(Xh))
    assert info.status == 0 and info.passes == idv.passes and info.shifted == idv.shifted
    assert np.array_equal(Q.numpy(), Qd) and np.array_equal(R.numpy(), Rd)


@pytest.mark.parametrize("n,precision", [(32, scqr3.PREC_FP64), (64, scqr3.PREC_FP64),
                                         (128, scqr3.PREC_FP64), (256, scqr3.PREC_FP64),
                                         (64, scqr3.PREC_MIXED)])
def test_chunked_first_gram(n, precision):
    m = 600_001  # chunks of 262,144 rows: 3, the last one ragged
    Xh = testmat(m, n, 1e8, seed=5100 + n)
    Qd, Rd, idv = device_run(Xh, precision=precision)
    Q, R, info = scqr3.factor_host(pinned(Xh), precision=precision)
    assert info.status == 0 and info.passes == idv.passes
    Q, R = Q.numpy(), R.numpy()
    assert np.linalg.norm(R - Rd) / np.linalg.norm(Rd) < 1e-12
    assert np.linalg.norm(Q.T @ Q - np.eye(n), 2) < 1e-13
    assert np.linalg.norm(Xh - Q @ R) / np.linalg.norm(Xh) < (1e-13 if precision == scqr3.PREC_FP64 else 1e-12)


def test_mixed_single_chunk_bitwise():
    Xh = testmat(200000, 128, 1e10, seed=5200)
    Qd, Rd, _ = device_run(Xh, precision=scqr3.PREC_MIXED)
    Q, R, info = scqr3.factor_host(pinned(Xh), precision=scqr3.PREC_MIXED)
    assert info.status == 0
    assert np.array_equal(Q.numpy(), Qd) and np.array_equal(R.numpy(), Rd)


def test_oblique_forms_are_bitwise_equal_at_any_size():
    m, n = 600000, 32
    Xh = testmat(m, n, 1e10, seed=5300)
    Bb = torch.from_numpy(block_diag_spd(m, 8, seed=5301)).cuda()
    Qd, Rd, _ = device_run(Xh, Bb)
    Q, R, info = scqr3.factor_host(pinned(Xh), Bb)
    assert info.status == 0
    assert np.array_equal(Q.numpy(), Qd) and np.array_equal(R.numpy(), Rd)
    Bc = scqr3.CsrB.from_arrays(laplacian_csr((600, 1000), 1e3))
    Qd, Rd, _ = device_run(Xh, Bc)
    Q, R, info = scqr3.factor_host(pinned(Xh), Bc)
    assert info.status == 0
    assert np.array_equal(Q.numpy(), Qd) and np.array_equal(R.numpy(), Rd)


@pytest.mark.parametrize("precision", [scqr3.PREC_FP64, scqr3.PREC_MIXED])
def test_alg2_stop_copies_the_last_iterate(precision):
    """Alg. 2 ends on its test after a solve that was followed by a Gram step:
    no chunked final solve, Q is copied whole (mixed: after the FP64 finish)."""
    Xh = testmat(100000, 64, 1e5, seed=5400)  # kappa^2 u ~ 1e-6: CholeskyQR2, two passes
    Qd, Rd, idv = device_run(Xh, algorithm=scqr3.ALG_ADAPTIVE, precision=precision)
    Q, R, info = scqr3.factor_host(pinned(Xh), algorithm=scqr3.ALG_ADAPTIVE, precision=precision)
    assert info.status == 0 and info.passes == idv.passes == 2
    assert np.array_equal(Q.numpy(), Qd) and np.array_equal(R.numpy(), Rd)


def test_in_place_strided_and_pageable():
    n = 48
    wide = testmat(200000, n + 16, 1e6, seed=5500)  # one chunk: bitwise comparable
    Xh = wide[:, :n]  # leading dimension n + 16
    Qd, Rd, _ = device_run(np.ascontiguousarray(Xh))
    T = torch.from_numpy(wide.copy())  # pageable, in place, ld = n + 16
    Xv = T[:, :n]
    Q, R, info = scqr3.factor_host(Xv, Q=Xv)
    assert info.status == 0
    assert np.array_equal(Xv.numpy(), Qd) and np.array_equal(R.numpy(), Rd)
    assert np.array_equal(T[:, n:].numpy(), wide[:, n:])  # columns past n untouched


def test_failure_status_and_q():
    Xh = testmat(5000, 16, 1e4, seed=5600)
    Xh[123, 5] = np.nan
    Q, R, info = scqr3.factor_host(pinned(Xh))
    assert info.status == scqr3.E_NONFINITE
    assert np.array_equal(np.isnan(Q.numpy()), np.isnan(Xh))  # pass 1 failed: Q holds X


def test_repeated_calls_reuse_workspace():
    Xh = testmat(400000, 64, 1e10, seed=5700)
    ws = scqr3.HostWorkspace(400000, 64)
    X = pinned(Xh)
    Q = torch.empty_like(X).pin_memory()
    R = torch.empty((64, 64), dtype=torch.float64)
    outs = []
    for _ in range(3):
        scqr3.factor_host(X, Q=Q, R=R, workspace=ws)
        outs.append((Q.numpy().copy(), R.numpy().copy()))
    assert all(np.array_equal(a[0], outs[0][0]) and np.array_equal(a[1], outs[0][1]) for a in outs)
