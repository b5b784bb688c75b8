"""The a-priori error bound of the low-precision matrix formats, checked on the CPU.

The GPU tests assert that the reconstruction from BF16 / E4M3 codes stays within
an element-wise bound of the float32 matrix's product.  Here that bound is
checked against a float32 computation written out step by step (codes decoded,
products and sums rounded to float32 one at a time, row scale last), and shown
to reject a planted mistake: a row scale off by a factor of two.
"""
import numpy as np
import pytest

from oracle import quantize_rows, stored_matrix
from parity_util import a_priori_bound


def float32_reconstruction(codes, scale, fmt, s):
    """Sequential float32 sums of code * s per row, then times the row scale."""
    q = stored_matrix(codes, fmt, None).astype(np.float32)      # decoded codes, exact in float32
    s32 = np.asarray(s, np.float32)
    acc = np.zeros(q.shape[0], np.float32)
    for j in range(q.shape[1]):
        acc = (acc + q[:, j] * s32[j]).astype(np.float32)
    return (acc * np.asarray(scale, np.float32)).astype(np.float64)


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_bound_holds_for_float32_arithmetic_and_rejects_a_wrong_scale(fmt):
    rng = np.random.default_rng(7)
    na, ns = 64, 700
    M = (rng.standard_normal((na, ns)) * 1e-3).astype(np.float32)
    M[3, :5] = [1e-9, -2e-9, 3e-12, 0.0, 5e-10]           # entries in E4M3's subnormal range
    s = rng.normal(0, 1.0, ns).astype(np.float32)
    codes, scale = quantize_rows(M, fmt)
    y = float32_reconstruction(codes, scale, fmt, s)
    y_true = M.astype(np.float64) @ s.astype(np.float64)
    bound = a_priori_bound(M, codes, scale, fmt, s, nterms=ns)
    assert np.all(np.abs(y - y_true) <= bound)
    # the largest row (relative to its bound) with its scale halved leaves the bound
    r = int(np.argmax(np.abs(y_true) / bound))
    bad = scale.copy()
    bad[r] *= np.float32(0.5)
    y_bad = float32_reconstruction(codes, bad, fmt, s)
    err = np.abs(y_bad - y_true)
    assert err[r] > bound[r]
    assert np.all(np.delete(err <= bound, r))
