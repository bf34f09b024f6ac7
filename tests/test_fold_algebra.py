"""The even / odd structure of the anti-reflective transform that the folded
tensor-core products rest on (CPU; the GPU parity of the folded products is in
tests/test_gpu_gemm_transform.py).

hat-S_n = diag(1, S_{n-2}, 1) with S_{n-2} the orthonormal DST-I (Sec. 3.2,
eqs. (lambda), (hats)); the oracle's transform_matrix builds it. Facts used:

* hat-S is symmetric, and each sine row k = 1..n-2 is even or odd about the
  middle: hat-S[k, n-1-j] = (-1)^(k+1) hat-S[k, j], because
  sin(pi k (n-1-j) / (n-1)) = (-1)^(k+1) sin(pi k j / (n-1)).
* So for even n, with s_j = x_j + x_{n-1-j} and d_j = x_j - x_{n-1-j}
  (j = 0..n/2-1), the odd-k rows need only s and the even-k rows only d:
  half the multiply-adds per output. The border rows 0 and n-1 are unit
  vectors (they read x_0 and x_{n-1}, kept in slot 0 of each half).
* The grouped row order puts the border row 0 and the odd rows first
  (0, 1, 3, ..., n-3) and the border row n-1 and the even rows after
  (n-1, n-2, n-4, ..., 2), so that a tile of 128 rows (n a multiple of 256)
  lies in one group and reads one half. Applying the transform twice
  (hat-S^2 = I) through the grouped halves recovers x.
"""
import numpy as np
import pytest

import oracle as O


def nat_of(p, n):
    """Natural row index of position p in the grouped order."""
    h = n // 2
    if p < h:
        return 0 if p == 0 else 2 * p - 1
    a = p - h
    return n - 1 if a == 0 else n - 2 * a


def folded_apply(x, n):
    """hat-S x computed from half-length products on the sums / differences of mirror pairs, rows
    produced in the grouped order and scattered back to their natural index."""
    S = O.transform_matrix(n, O.AR)
    h = n // 2
    s = x[:h] + x[::-1][:h]          # s_j = x_j + x_{n-1-j}
    d = x[:h] - x[::-1][:h]
    s[0], d[0] = x[0], x[n - 1]      # slot 0: the raw endpoints (border rows read them alone)
    y = np.empty(n)
    for p in range(n):
        k = nat_of(p, n)
        if k in (0, n - 1):
            y[k] = s[0] if k == 0 else d[0]
            continue
        half = S[k, :h].copy()
        half[0] = 0.0                # sine rows vanish on the border columns
        y[k] = half @ (s if k % 2 == 1 else d)
    return y


@pytest.mark.parametrize("n", [6, 10, 256, 512])
def test_sine_rows_are_even_or_odd_about_the_middle(n):
    S = O.transform_matrix(n, O.AR)
    np.testing.assert_allclose(S, S.T, atol=1e-15)
    for k in range(1, n - 1):
        np.testing.assert_allclose(S[k, ::-1], (-1) ** (k + 1) * S[k], atol=1e-14)
    np.testing.assert_array_equal(S[0], np.eye(n)[0])
    np.testing.assert_array_equal(S[n - 1], np.eye(n)[n - 1])


@pytest.mark.parametrize("n", [6, 10, 256, 512])
def test_grouped_order_is_a_permutation_with_one_parity_per_half(n):
    rows = [nat_of(p, n) for p in range(n)]
    assert sorted(rows) == list(range(n))
    first, second = rows[: n // 2], rows[n // 2:]
    assert first[0] == 0 and all(k % 2 == 1 for k in first[1:])
    assert second[0] == n - 1 and all(k % 2 == 0 for k in second[1:])
    if n % 256 == 0:                 # 128-row tiles never straddle the two groups
        assert all((t * 128 < n // 2) == (t * 128 + 127 < n // 2) for t in range(n // 128))


@pytest.mark.parametrize("n", [6, 10, 256, 512])
def test_folded_halves_reproduce_the_transform(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n)
    S = O.transform_matrix(n, O.AR)
    np.testing.assert_allclose(folded_apply(x, n), S @ x, atol=1e-12)
    np.testing.assert_allclose(folded_apply(folded_apply(x, n), n), x, atol=1e-12)   # hat-S^2 = I
