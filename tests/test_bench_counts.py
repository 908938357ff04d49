"""The algorithmic byte counts behind the roofline numbers bench.py reports
(no GPU): the persistent CG's bytes per row-iteration (couplings, column
indices, vector accesses) and the batched engine's bytes per row-pass, at the
values quoted with the measurements."""
import pytest

import bench


@pytest.mark.parametrize("nphi,cb,vb,pre,expected", [
    (10, 4, 4, False, 201.6),               # p = 3, FP32: the headline kernel
    (10, 4, 4, True, 249.6),                # p = 3, FP32, block-Jacobi (A P couplings + row of P)
    (6, 4, 4, False, 96 + 16 / 6 + 40),     # p = 2, FP32: 138.67
    (15, 4, 4, False, 240 + 16 / 15 + 40),  # p = 4, FP32: 281.07
    (6, 2, 4, False, 48 + 16 / 6 + 40),     # p = 2, BF16 couplings: 90.67
    (10, 8, 8, False, 320 + 1.6 + 80),      # p = 3, FP64
])
def test_cg_bytes_per_row_iteration(nphi, cb, vb, pre, expected):
    assert bench.bytes_per_row_iter(nphi, cb, vb, precond=pre) == pytest.approx(expected, rel=1e-12)


def test_engine_bytes_share_the_couplings():
    # R right-hand sides share one coupling stream: per RHS the bytes fall toward 40 B
    one = bench.engine_bytes_per_row_pass(10, 4, 1)
    eight = bench.engine_bytes_per_row_pass(10, 4, 8)
    assert one == pytest.approx(160 + 1.6 + 40)
    assert eight / 8 == pytest.approx((160 + 1.6) / 8 + 40)
