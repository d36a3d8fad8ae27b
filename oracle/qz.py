"""Eigenvalue (linearisation + QZ) root finder of the 2-bounce resultant
(TEST INFRASTRUCTURE: a completeness reference for the bisection solver).

Only ``tests/`` and ``bench.py``'s CPU legs may import this module; the
product path never does.  It shares no code with the CUDA library.

Sec. 4.2 ("Discussion") names the alternative to bisection on the sign of
det R(v1): linearise the matrix polynomial R(v1) and solve the generalised
eigenvalue problem by the QZ decomposition, which finds every zero of the
determinant without sampling.  This module states it in plain numpy/scipy
FP64:

1. R(v1) = sum_k R_k v1^k, the Bezout matrix of Eq. eq_bezout with
   polynomial entries: B_ij = sum_{k=0}^{min(i, n-1-j)} (A_{i-k} B_{j+1+k} -
   B_{i-k} A_{j+1+k}) where A_m(v1), B_m(v1) are the u1^m coefficients of the
   system's a and b (products of polynomials in v1);
2. the companion pencil of size n d (d the v1-degree of R):
       A = [[0, I, 0, ...], ..., [0, ..., 0, I], [-R_0, -R_1, ..., -R_{d-1}]]
       B = diag(I, ..., I, R_d),
   whose generalised eigenvalues are the zeros of det R(v1) (eigenvalues at
   infinity come from a singular R_d and are dropped);
3. the real eigenvalues in [0, 1] (imaginary part below 1e-6 of
   max(1, |v1|)) are the candidate roots v1*.

The path phase after the roots is the bisection oracle's own (u1 from
a(u1, v1*) = 0, the mapping, path-space Newton, checks), so the two solvers
differ only in how they find v1*.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

IMAG_TOL = 1e-6
DOMAIN_SLACK = 1e-9


def _pmul(p, q):
    return np.convolve(p, q)


def _padd(p, q):
    n = max(p.size, q.size)
    r = np.zeros(n)
    r[:p.size] += p
    r[:q.size] += q
    return r


def bezout_matrix_poly(a, b, da, db):
    """R(v1) as an array [d + 1, n, n] of coefficient matrices (Eq. eq_bezout,
    explicit sum), n = max(da, db).  a, b: bivariate coefficient arrays
    c[i, j] of u1^i v1^j."""
    n = max(da, db)
    A = [np.asarray(a[m], float) if m <= da else np.zeros(1) for m in range(n + 1)]
    B = [np.asarray(b[m], float) if m <= db else np.zeros(1) for m in range(n + 1)]
    ent = [[np.zeros(1) for _ in range(n)] for _ in range(n)]
    for i in range(n):
        for j in range(n):
            acc = np.zeros(1)
            for k in range(min(i, n - 1 - j) + 1):
                acc = _padd(acc, _padd(_pmul(A[i - k], B[j + 1 + k]), -_pmul(B[i - k], A[j + 1 + k])))
            ent[i][j] = acc
    d = max(e.size for row in ent for e in row) - 1
    R = np.zeros((d + 1, n, n))
    for i in range(n):
        for j in range(n):
            R[:ent[i][j].size, i, j] = ent[i][j]
    return R


def matrix_poly_eigenvalues(R):
    """Finite generalised eigenvalues of the companion pencil of R (QZ)."""
    R = np.asarray(R, float)
    # drop leading coefficient matrices that vanish exactly
    while R.shape[0] > 1 and not np.any(R[-1]):
        R = R[:-1]
    d, n = R.shape[0] - 1, R.shape[1]
    if d == 0:
        return np.zeros(0, complex)
    # one common scale for every coefficient matrix (the eigenvalues are
    # unchanged)
    scale = max(np.max(np.abs(R)), 1e-300)
    R = R / scale
    N = n * d
    A = np.zeros((N, N))
    Bm = np.eye(N)
    for k in range(d - 1):
        A[k * n:(k + 1) * n, (k + 1) * n:(k + 2) * n] = np.eye(n)
    for k in range(d):
        A[(d - 1) * n:, k * n:(k + 1) * n] = -R[k]
    Bm[(d - 1) * n:, (d - 1) * n:] = R[d]
    alpha, beta = scipy.linalg.eig(A, Bm, right=False, homogeneous_eigvals=True)
    fin = np.abs(beta) > 1e-14 * np.maximum(np.abs(alpha), 1e-300)
    return alpha[fin] / beta[fin]


def v_roots(a, b, da, db, lo=0.0, hi=1.0):
    """Real zeros of det R(v1) in [lo, hi] by linearisation + QZ, sorted."""
    lam = matrix_poly_eigenvalues(bezout_matrix_poly(a, b, da, db))
    re = lam.real
    ok = (np.abs(lam.imag) <= IMAG_TOL * np.maximum(1.0, np.abs(re))) & (re >= lo - DOMAIN_SLACK) & \
        (re <= hi + DOMAIN_SLACK)
    return np.sort(np.clip(re[ok], lo, hi))
