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
