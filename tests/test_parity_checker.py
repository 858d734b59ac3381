"""The parity checker itself (tests/gpu_common.py), on the CPU: every GPU-vs-oracle
comparison goes through check_close and check_fd, so their semantics are pinned here
with hand-made arrays whose per-entry and norm errors are known exactly."""

import numpy as np
import pytest

from gpu_common import check_close, check_fd, entry_err, rel_err


def test_equal_fields_pass_with_zero_error():
    b = np.linspace(-1.0, 2.0, 1000)
    assert check_close(b.copy(), b, 1e-12) == (0.0, 0.0)


def test_one_bad_entry_fails_although_the_norm_passes():
    # 10^4 entries of 1, one of them off by 5e-12: the norm error is 5e-14 (below
    # 1e-12), the per-entry error 5e-12 (above): the per-entry bound must catch it
    b = np.ones(10000)
    a = b.copy()
    a[1234] += 5e-12
    assert rel_err(a, b) < 1e-12
    assert entry_err(a, b) == pytest.approx(5e-12, rel=1e-3)
    with pytest.raises(AssertionError, match="per-entry"):
        check_close(a, b, 1e-12)


def test_entries_are_scaled_by_the_largest_reference_entry():
    # the bound is tol * max|b|: an error of 1e-13 on a small entry passes when the
    # largest entry is 1, and fails when every entry is small
    err = np.array([0.0, 1e-13, 0.0])
    b = np.array([1.0, 1e-3, -0.5])
    check_close(b + err, b, 1e-12)                 # 1e-13 / 1
    small = b * 1e-3
    with pytest.raises(AssertionError):
        check_close(small + err, small, 1e-12)     # 1e-13 / 1e-3


def test_non_finite_entries_fail():
    b = np.ones(8)
    a = b.copy()
    a[3] = np.nan
    with pytest.raises(AssertionError, match="non-finite"):
        check_close(a, b, 1e-3)


def test_the_mask_selects_the_compared_entries():
    # populations (Q, N): a wrong value on a masked-out (solid) node is not compared
    b = np.ones((3, 5))
    a = b.copy()
    a[:, 2] = 7.0
    mask = np.array([True, True, False, True, True])
    assert check_close(a, b, 1e-12, mask) == (0.0, 0.0)
    with pytest.raises(AssertionError):
        check_close(a, b, 1e-12)


def test_fd_check_is_relative_per_entry_with_a_floor():
    check_fd(1.0, 1.0 + 0.9e-4, 1e-4, 0.0)
    with pytest.raises(AssertionError):
        check_fd(1.0, 1.0 + 1.1e-4, 1e-4, 0.0)
    # a tiny gradient entry passes within the stated floor, not without it
    check_fd(1e-15, 3e-15, 1e-4, 1e-14)
    with pytest.raises(AssertionError):
        check_fd(1e-15, 3e-15, 1e-4, 0.0)
