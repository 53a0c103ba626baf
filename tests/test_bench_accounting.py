"""Host-side checks of bench.py's accounting for the tensor-core substitution:
the launches it attributes per pass must be the ones the library makes
(block width 16 for n <= 64, 32 above; one update launch per 32 columns right
of each diagonal block), and the FP64 flops of the diagonal blocks must add
up to the blocked substitution's count."""
import os
import sys

import pytest

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
import bench  # noqa: E402


def library_launches(n):
    """The loop of the library's tensor-core substitution, restated."""
    w = 16 if n <= 64 else 32
    nb = (n + w - 1) // w
    solves, updates = [], []
    for J in range(nb):
        solves.append(min(w, n - w * J))
        c0 = w * (J + 1)
        while c0 < n:
            updates.append((w, min(32, n - c0)))
            c0 += 32
    return solves, updates


@pytest.mark.parametrize("n", [1, 16, 17, 32, 33, 48, 63, 64, 65, 96, 100, 127, 128])
def test_update_launches_match_the_library(n):
    solves, updates = library_launches(n)
    assert bench.tc_update_cols(n) == updates
    assert bench.tc_block_width(n) == (16 if n <= 64 else 32)
    assert sum(solves) == n


def test_headline_launch_shapes():
    assert bench.tc_update_cols(64) == [(16, 32), (16, 16), (16, 32), (16, 16)]
    assert bench.tc_update_cols(128) == [(32, 32)] * 6
    assert bench.tc_update_cols(32) == [(16, 16)]


@pytest.mark.parametrize("n", [32, 64, 100, 128])
def test_block_flops_sum(n):
    """Per pass the diagonal blocks do sum_J w_J^2 flops per row (w_J (w_J - 1)/2
    FMAs and w_J multiplies each), against n^2 for the unblocked substitution."""
    from paper_1809_11085_gb300 import scqr3

    m, passes = 1000, 3
    solves, _ = library_launches(n)
    got = sum(bench.pass_kernel_flops(m, n, scqr3.KERNEL_PASS, 0, passes, gram_in_pass=False, block=J)
              for J in range(len(solves)))
    assert got == m * sum(w * w for w in solves)
    assert got <= m * n * n
    # a skipped pass does no work
    assert bench.pass_kernel_flops(m, n, scqr3.KERNEL_PASS, passes, passes, gram_in_pass=False, block=0) == 0


def test_update_roofline_bytes():
    r = bench.tc_update_roofline(1 << 20, 64, [(1.0, (16, 32)), (0.5, (16, 16))])
    # mean bytes per launch: (16 + 64) * 8 and (16 + 32) * 8 per row
    assert r["bytes_per_launch"] == (1 << 20) * 8 * (80 + 48) / 2
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"


def fused_ops_restated(n):
    """FP64-pipe operations per row of the one-sweep substitution, counted from
    its structure: NP / 16 diagonal blocks of 16 columns (16 * 15 / 2 FMAs and 16
    multiplies each) and one subtraction per entry an off-diagonal product
    updates (NP = 64: x_1 by y_0, x_2 and x_3 by [y_0 y_1], x_3 by y_2)."""
    np_ = 32 if n <= 32 else 64
    blocks = np_ // 16
    updated = {32: [16], 64: [16, 16, 16, 16]}[np_]
    return blocks * (16 * 15 // 2 + 16) + sum(updated)


@pytest.mark.parametrize("n", [17, 32, 33, 64])
def test_fused_fp64_ops(n):
    assert bench.fused_fp64_ops(n) == fused_ops_restated(n)
    assert bench.fused_fp64_ops(64) == 608
    # a quarter-plus of the unblocked substitution's n^2 FP64 flops per row
    assert bench.fused_fp64_ops(64) < 64 * 64 // 6


def test_fused_used_range():
    from paper_1809_11085_gb300 import scqr3

    assert [n for n in (16, 17, 64, 65) if bench.fused_used(scqr3.PREC_TC, n)] == [17, 64]
    assert not bench.fused_used(scqr3.PREC_FP64, 64) and not bench.fused_used(scqr3.PREC_MIXED_TC, 64)


def test_exact_r_of_the_generator():
    """exact_r(s, V) is the R factor of X = U diag(s) V^T for any orthonormal U:
    it matches numpy's Householder R of such an X (signs fixed) to rounding."""
    import numpy as np

    from paper_1809_11085_gb300.testmat import testmat_factors

    U, s, V = testmat_factors(3000, 12, 1e6, seed=5)
    X = (U * s) @ V.T
    _, Rn = np.linalg.qr(X)
    Rn = Rn * np.sign(np.diag(Rn))[:, None]
    Re = bench.exact_r(s, V)
    assert np.all(np.diag(Re) > 0) and np.allclose(np.tril(Re, -1), 0)
    assert np.linalg.norm(Re - Rn) / np.linalg.norm(Rn) < 1e-12
