"""Exact rational brute force for tiny pulsars.  TEST INFRASTRUCTURE ONLY.

With rational TOAs, residuals, noise levels and prior, and no signal, the dense
covariance of the model (see ``dense.py``) is a rational matrix, so both parts
of the Gaussian log-density, det C and r^T C^-1 r, are exact rationals.  The
Kalman filter's prediction-error decomposition must reproduce them:
prod_k S_k = det C and sum_k e_k^2 / S_k = r^T C^-1 r.
"""
from __future__ import annotations

from fractions import Fraction as Fr


def covariance(t, sig2, p0, R):
    t = [Fr(x) for x in t]
    tau = [x - t[0] for x in t]
    n = len(t)
    C = [[Fr(0)] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            m, M = min(tau[i], tau[j]), max(tau[i], tau[j])
            C[i][j] = (Fr(p0[0]) + Fr(p0[1]) * (tau[i] + tau[j]) + Fr(p0[2]) * tau[i] * tau[j]
                       + Fr(sig2) * (m * m * M / 2 - m ** 3 / 6))
        C[i][i] += Fr(R[i])
    return C


def det_and_quad(C, r):
    """(det C, r^T C^-1 r) by exact Gaussian elimination."""
    n = len(C)
    A = [row[:] + [Fr(x)] for row, x in zip(C, r)]
    det = Fr(1)
    for k in range(n):
        piv = next(i for i in range(k, n) if A[i][k] != 0)
        if piv != k:
            A[k], A[piv] = A[piv], A[k]
            det = -det
        det *= A[k][k]
        for i in range(k + 1, n):
            f = A[i][k] / A[k][k]
            for j in range(k, n + 1):
                A[i][j] -= f * A[k][j]
    # back substitution for x = C^-1 r
    x = [Fr(0)] * n
    for i in reversed(range(n)):
        x[i] = (A[i][n] - sum(A[i][j] * x[j] for j in range(i + 1, n))) / A[i][i]
    quad = sum(Fr(ri) * xi for ri, xi in zip(r, x))
    return det, quad
