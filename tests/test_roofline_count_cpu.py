"""The roofline numerator of the benchmark line: bench.gj_inverse_flops, the
algorithmic flops of the blocked Gauss-Jordan inverse of the core, checked
against a blocked Gauss-Jordan inversion run in numpy that counts the
multiply-adds of every product it performs and whose result is checked
against the inverse.

Each sweep k with panel width w maps A to B with pivot block P = A[k,k]:
B[k,k] = P^{-1} (w^3); B[k,j] = P^{-1} A[k,j]; B[i,k] = -A[i,k] P^{-1};
B[i,j] = A[i,j] - A[i,k] B[k,j] (i, j outside the panel).  A leading
identity block of `ident` rows (rounded down to whole panels) is eliminated
in one step, which needs only the trailing update.
"""
import numpy as np
import pytest

import bench


def _counted_gj_inverse(A, ident, b):
    n = A.shape[0]
    A = A.copy()
    nt = (n + b - 1) // b
    k0 = min(ident // b, nt - 1)
    e = k0 * b
    fma = 0
    if e:                                    # identity pivot: B[i,j] -= A[i,k] A[k,j]
        L, Rr = A[e:, :e].copy(), A[:e, e:].copy()
        A[e:, e:] -= L @ Rr
        fma += L.shape[0] * L.shape[1] * Rr.shape[1]
        A[e:, :e] = -L
    for k in range(k0, nt):
        r0, r1 = k * b, min(n, (k + 1) * b)
        w = r1 - r0
        out = np.r_[0:r0, r1:n]
        Pinv = np.linalg.inv(A[r0:r1, r0:r1])
        fma += w ** 3
        row = Pinv @ A[r0:r1][:, out]                      # B[k, j]
        col = A[out][:, r0:r1]
        A[np.ix_(out, out)] -= col @ row                    # B[i, j]
        A[np.ix_(out, np.arange(r0, r1))] = -col @ Pinv     # B[i, k]
        fma += w * w * len(out) + len(out) * len(out) * w + len(out) * w * w
        A[np.ix_(np.arange(r0, r1), out)] = row
        A[r0:r1, r0:r1] = Pinv
    return A, fma


@pytest.mark.parametrize("n,ident,b", [(1200, 400, 64), (300, 0, 64), (250, 25, 64), (130, 64, 32),
                                       (75, 25, 16), (64, 0, 64)])
def test_gj_inverse_flops_counts_the_blocked_inversion(n, ident, b):
    rng = np.random.default_rng(n + ident)
    X = rng.standard_normal((n, n))
    X = 0.5 * (X + X.T)
    A = np.eye(n) + 0.3 * X / np.linalg.norm(X, 2)
    e = min(ident // b, (n + b - 1) // b - 1) * b
    A[:e, :e] = np.eye(e)
    inv, fma = _counted_gj_inverse(A, ident, b)
    assert np.linalg.norm(inv @ A - np.eye(n)) < 1e-10 * n
    assert 2 * fma == bench.gj_inverse_flops(n, ident, b)
