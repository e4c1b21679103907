"""Precision of the tensor-core factorisation schedule, on the CPU.

The float32 kernels with hydrodynamic interaction factor the RPY tensor W
(Eqs. 2-3) with the trailing updates on the tensor cores, which read their
operands as tf32 (ten stored mantissa bits). Each float32 product x y of
those updates is formed there as hi(x) hi(y) + hi(x) lo(y) + lo(x) hi(y),
hi the tf32 truncation of x and lo = x - hi, itself read as tf32. This test
runs the kernel's schedule in numpy - the head columns (t0 = 3 max(0, N - 42)
rows) factored and solved in float32, the trailing block updated with their
outer product, then 32-column panels of the trailing block, each diagonal
block factored and the rows below solved in float32 and the rest of the
block updated - on the oracle's tensor of collapsed-chain and vWF-chain
conformations, and
compares the factor with the float64 Cholesky factor of the same tensor:

- with three tf32 products the factor has float32-class accuracy (about
  2.5e-7 of the largest entry, within five times the error of a plain
  float32 Cholesky factor, about 1e-7: the dropped lo lo term and the tf32
  reading of lo cost a few ulps);
- with one tf32 product (plain tf32 operands) it is off by about 4e-4,
  above the 1e-4 tolerance of the float32 runs at every size: the reason
  the kernel spends three MMAs per product.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2206_05851_gb300 import inputs as I


def _tf32(x):
    """Truncation to tf32 (the low 13 mantissa bits cleared), as the tensor
    cores read a 32-bit operand."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return u.view(np.float32)


def _outer_update(T, X, split):
    """T - X X^T in float32, the products formed the tensor-core way: per
    K step of 8 the tf32 products summed exactly and added to the float32
    accumulator (split: hi hi + hi lo + lo hi; else hi hi only)."""
    hi = _tf32(X)
    lo = _tf32(X - hi)
    acc = T.astype(np.float32).copy()
    for k0 in range(0, X.shape[1], 8):
        h = hi[:, k0:k0 + 8].astype(np.float64)
        p = h @ h.T
        if split:
            l = lo[:, k0:k0 + 8].astype(np.float64)
            p += h @ l.T + l @ h.T
        acc = (acc - p).astype(np.float32)
    return acc


def _chol32(A):
    """Plain float32 column Cholesky of a small block (lower factor)."""
    A = A.astype(np.float32).copy()
    n = A.shape[0]
    L = np.zeros_like(A)
    for k in range(n):
        d = np.float32(A[k, k]) - np.float32(np.dot(L[k, :k], L[k, :k]))
        L[k, k] = np.sqrt(d, dtype=np.float32)
        for i in range(k + 1, n):
            L[i, k] = (A[i, k] - np.float32(np.dot(L[i, :k], L[k, :k]))) / L[k, k]
    return L


def _solve32(B, L):
    """X L^T = B in float32 (forward substitution over the columns)."""
    X = B.astype(np.float32).copy()
    for k in range(L.shape[0]):
        X[:, k] = (X[:, k] - X[:, :k] @ L[k, :k]) / L[k, k]
    return X


def _tc_schedule(W, N, split):
    n = 3 * N
    t0 = 3 * max(0, N - 42)
    W = W.astype(np.float32)
    L = np.zeros((n, n), dtype=np.float32)
    T = W[t0:, t0:].copy()
    if t0:
        L[:t0, :t0] = _chol32(W[:t0, :t0])
        X = _solve32(W[t0:, :t0], L[:t0, :t0])
        L[t0:, :t0] = X
        T = _outer_update(T, X, split)
    m = n - t0
    for c0 in range(0, m, 32):
        c1 = min(c0 + 32, m)
        Ld = _chol32(T[c0:c1, c0:c1])
        L[t0 + c0:t0 + c1, t0 + c0:t0 + c1] = Ld
        if c1 < m:
            X = _solve32(T[c1:, c0:c1], Ld)
            L[t0 + c1:, t0 + c0:t0 + c1] = X
            T[c1:, c1:] = _outer_update(T[c1:, c1:], X, split)
    return L


def _conformation(N, seed, vwf=False):
    ch = I.vwf_chain(2, n_beads=N) if vwf else I.collapsed_chain(2, n_beads=N)
    return I.initial_positions(I.custom([ch], 1e-5, 10, 10), seed=seed)


@pytest.mark.parametrize("N,seed,vwf", [(12, 1, False), (20, 8, False), (33, 2, False), (42, 7, False),
                                        (43, 3, False), (50, 4, False), (50, 5, False), (50, 6, True)])
def test_three_tf32_products_keep_float32_accuracy(N, seed, vwf):
    W = O.rpy_matrix(1.0, _conformation(N, seed, vwf))
    L64 = np.linalg.cholesky(W)
    scale = np.abs(L64).max()
    e32 = np.abs(_chol32(W).astype(np.float64) - L64).max() / scale
    e3 = np.abs(_tc_schedule(W, N, True).astype(np.float64) - L64).max() / scale
    e1 = np.abs(_tc_schedule(W, N, False).astype(np.float64) - L64).max() / scale
    assert e3 <= 5.0 * e32 and e3 <= 1e-6, (e3, e32)
    assert e1 > 1e-4 and e1 >= 100.0 * e3, (e1, e3)
