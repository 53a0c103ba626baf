"""scqr3_factor_noalloc: the factorization for callers that cannot allocate
device memory (an application that owns all device memory through its own
pool, a caller at the edge of the memory limit, a C/Fortran code with no
device allocator). It must give the same Q and R as scqr3_factor, call after
call, although every call reuses the same fixed scratch array inside the
library; and it must refuse problems that need more scratch than that array.

Kept in a file of its own that pytest collects last, so that a failure here
does not hide the other tests."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1809_11085_gb300 import scqr3  # noqa: E402
from paper_1809_11085_gb300.testmat import testmat  # noqa: E402

pytestmark = pytest.mark.gpu
E_SCRATCH_LIMIT = -107


def _fn():
    from paper_1809_11085_gb300 import build

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = scqr3.lib().scqr3_factor_noalloc
    p = ctypes.c_void_p
    f.argtypes = [p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, p, ctypes.c_int64, p, p, p]
    f.restype = ctypes.c_int
    return f


def _call(f, X, Q, R, info):
    m, n = X.shape
    stream = torch.cuda.current_stream().cuda_stream
    return f(X.data_ptr(), m, n, X.stride(0), Q.data_ptr(), Q.stride(0), R.data_ptr(),
             info.data_ptr(), ctypes.c_void_p(stream))


def test_noalloc_matches_scqr3_factor_on_two_calls_in_a_row():
    f = _fn()
    m, n = 20000, 32
    Xh = testmat(m, n, 1e6, seed=4242)
    X = torch.from_numpy(Xh).cuda()
    Q0, R0, info0 = scqr3.factor(X)
    torch.cuda.synchronize()
    assert info0.status == 0
    Q0h, R0h = Q0.cpu().numpy(), R0.cpu().numpy()
    info = torch.zeros(scqr3.INFO_BYTES, dtype=torch.uint8, device="cuda")
    for call in range(2):
        Q = torch.full_like(X, float("nan"))
        R = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(f, X, Q, R, info) == 0
        torch.cuda.synchronize()
        inf = scqr3.Info.from_bytes(info.cpu().numpy().tobytes())
        assert inf.status == 0 and inf.passes == info0.passes, (call, inf)
        Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
        # same tolerances as the parity tests (kappa <= 1e8)
        assert np.linalg.norm(Rh - R0h) / np.linalg.norm(R0h) <= 1e-12
        assert np.linalg.norm(Qh - Q0h) / np.linalg.norm(Q0h) <= 1e-12
        assert np.linalg.norm(Qh.T @ Qh - np.eye(n), 2) <= 1e-13
        assert np.linalg.norm(Xh - Qh @ Rh) / np.linalg.norm(Xh) <= 1e-13


def _check_against_factor(f, info, m, n, kappa, seed):
    Xh = testmat(m, n, kappa, seed=seed)
    X = torch.from_numpy(Xh).cuda()
    Q0, R0, info0 = scqr3.factor(X)
    torch.cuda.synchronize()
    assert info0.status == 0
    Q = torch.full_like(X, float("nan"))
    R = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    assert _call(f, X, Q, R, info) == 0
    torch.cuda.synchronize()
    inf = scqr3.Info.from_bytes(info.cpu().numpy().tobytes())
    assert inf.status == 0 and inf.passes == info0.passes, (m, n, inf)
    Qh, Rh, Q0h, R0h = Q.cpu().numpy(), R.cpu().numpy(), Q0.cpu().numpy(), R0.cpu().numpy()
    assert np.linalg.norm(Rh - R0h) / np.linalg.norm(R0h) <= 1e-12, (m, n)
    assert np.linalg.norm(Qh - Q0h) / np.linalg.norm(Q0h) <= 1e-12, (m, n)
    assert np.linalg.norm(Qh.T @ Qh - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(Xh - Qh @ Rh) / np.linalg.norm(Xh) <= 1e-13


def test_noalloc_shapes_in_sequence_share_the_array():
    """The shared array keeps what the last call left: the number of partial
    Gram slots and the padded n change from shape to shape, so calls of
    different shapes in a row must still match scqr3_factor each time (a stale
    entry read from a larger earlier call would show)."""
    f = _fn()
    info = torch.zeros(scqr3.INFO_BYTES, dtype=torch.uint8, device="cuda")
    for (m, n, seed) in ((200, 128, 1), (20000, 16, 2), (20011, 64, 3), (300, 100, 4), (20000, 16, 5)):
        _check_against_factor(f, info, m, n, 1e6, seed)


def test_noalloc_largest_shape_that_fits():
    """The largest m (n = 128) whose workspace fits the fixed array runs; one
    more panel of rows is refused."""
    f = _fn()
    n, limit = 128, 16 << 20
    lo, hi = n, 1 << 22
    assert scqr3.workspace_bytes(lo, n) <= limit < scqr3.workspace_bytes(hi, n)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if scqr3.workspace_bytes(mid, n) <= limit:
            lo = mid
        else:
            hi = mid
    info = torch.zeros(scqr3.INFO_BYTES, dtype=torch.uint8, device="cuda")
    _check_against_factor(f, info, lo, n, 1e4, 6)
    X = torch.zeros((hi, n), dtype=torch.float64, device="cuda")
    Q = torch.empty_like(X)
    R = torch.empty((n, n), dtype=torch.float64, device="cuda")
    assert _call(f, X, Q, R, info) == E_SCRATCH_LIMIT


def test_noalloc_argument_codes_follow_its_own_prototype():
    """-k names argument k of scqr3_factor_noalloc: X 1, ldx 4, Q 5, ldq 6,
    R 7, info 8."""
    f = _fn()
    m, n = 1000, 8
    X = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    Q = torch.empty_like(X)
    R = torch.empty((n, n), dtype=torch.float64, device="cuda")
    info = torch.zeros(scqr3.INFO_BYTES, dtype=torch.uint8, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    xp, qp, rp, ip = X.data_ptr(), Q.data_ptr(), R.data_ptr(), info.data_ptr()
    assert f(None, m, n, n, qp, n, rp, ip, s) == -1
    assert f(xp, m, n, n - 1, qp, n, rp, ip, s) == -4
    assert f(xp, m, n, n, None, n, rp, ip, s) == -5
    assert f(xp, m, n, n, qp, n - 1, rp, ip, s) == -6
    assert f(xp, m, n, n, qp, n, None, ip, s) == -7
    assert f(xp, m, n, n, qp, n, rp, None, s) == -8
    assert f(xp, m, 0, n, qp, n, rp, ip, s) == -3
    assert f(xp, n - 1, n, n, qp, n, rp, ip, s) == -2


def test_noalloc_rejects_problems_beyond_its_scratch():
    f = _fn()
    m, n = 200000, 128
    need = scqr3.workspace_bytes(m, n)
    assert need > (16 << 20)
    X = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    Q = torch.empty_like(X)
    R = torch.empty((n, n), dtype=torch.float64, device="cuda")
    info = torch.zeros(scqr3.INFO_BYTES, dtype=torch.uint8, device="cuda")
    assert _call(f, X, Q, R, info) == E_SCRATCH_LIMIT
