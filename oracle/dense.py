"""Dense helpers of the oracle for tiny inputs (TEST INFRASTRUCTURE ONLY).

Library primitives (numpy.linalg) serve as single steps; nothing here is
blocked, fused or reordered.
"""
import numpy as np


def to_dense(Q):
    n = int(Q["n"])
    A = np.zeros((n, n))
    rp, ci, v = Q["row_ptr"], Q["col"], Q["val"]
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            A[i, ci[p]] += v[p]
    return A


def step_constant_L(Q):
    """L = lambda_max(D^-1/2 Q D^-1/2), the smallest c with c*D - Q >= 0
    (rows with zero diagonal are left out: they are all-zero rows of an SPSD Q)."""
    A = to_dense(Q)
    d = np.diag(A).copy()
    keep = d > 0
    A = A[np.ix_(keep, keep)]
    s = 1.0 / np.sqrt(d[keep])
    M = A * s[:, None] * s[None, :]
    return float(np.linalg.eigvalsh(M)[-1])


def f_value(A, b, x):
    """f(x) = 1/2 <x, Q x> - <b, x>  (eq. qp)."""
    return 0.5 * x @ (A @ x) - b @ x
