"""Pins of the oracle's Gauss-Lobatto basis and LSERK4 coefficients.

The paper discretises on Legendre-Gauss-Lobatto nodes (Sec. 2.2) and
integrates with a fourth-order low-storage Runge-Kutta scheme (Sec. 4).
Closed forms and exactness properties below fix the nodes, weights,
derivative matrix and the scheme independently of the oracle's code."""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("N", [2, 3, 4])
def test_lgl_closed_forms(ora, N):
    x, w, D = ora.lgl(N)
    known = {
        2: ([-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
        3: ([-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
        4: ([-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
    }
    xs, ws = known[N]
    assert np.allclose(x, xs, atol=1e-15, rtol=0)
    assert np.allclose(w, ws, atol=1e-15, rtol=0)


@pytest.mark.parametrize("N", [1, 3, 5, 7, 9])
def test_lgl_quadrature_and_derivative_exactness(ora, N):
    x, w, D = ora.lgl(N)
    assert abs(w.sum() - 2.0) < 1e-14
    # Gauss-Lobatto quadrature is exact for degree <= 2N - 1
    for p in range(2 * N):
        exact = (1 - (-1) ** (p + 1)) / (p + 1)
        assert abs((w * x ** p).sum() - exact) < 1e-13
    # ... and not for degree 2N (the Lobatto rule's known defect)
    p = 2 * N
    assert abs((w * x ** p).sum() - 2.0 / (p + 1)) > 1e-6
    # D differentiates polynomials of degree <= N exactly
    for p in range(N + 1):
        d = D @ x ** p
        ref = p * x ** (p - 1) if p > 0 else 0 * x
        assert np.abs(d - ref).max() < 1e-11 * max(1, N ** 2)
    # interior nodes are roots of P_N'
    if N > 1:
        dP = np.polynomial.legendre.Legendre.basis(N).deriv()
        assert np.abs(dP(x[1:-1])).max() < 1e-12


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_summation_by_parts(ora, N):
    x, w, D = ora.lgl(N)
    Q = np.diag(w) @ D
    B = np.zeros((N + 1, N + 1)); B[0, 0] = -1; B[N, N] = 1
    assert np.abs(Q + Q.T - B).max() < 1e-13
    # D_00 = -N(N+1)/4 (so the split-form volume matrix 2D - B/w has zero corners)
    assert abs(D[0, 0] + N * (N + 1) / 4) < 1e-12
    assert abs(D[N, N] - N * (N + 1) / 4) < 1e-12


def _butcher_from_2n(A, B):
    """Butcher tableau of the 2N-storage scheme dU = A_s dU + dt f; U += B_s dU."""
    s = len(A)
    # stage s input: U_s = U0 + dt * sum_j a[s][j] f_j ; dU_s = sum_j g[s][j] f_j
    a = np.zeros((s + 1, s))
    g = np.zeros(s)
    for st in range(s):
        g = A[st] * g
        g[st] += 1.0
        a[st + 1] = a[st] + B[st] * g
    return a[:s], a[s]


def test_lserk4_order_conditions(ora):
    A, B, c = ora.lserk4()
    a, b = _butcher_from_2n(A, B)
    # stage times equal the row sums of the tableau
    assert np.abs(a.sum(1) - c).max() < 1e-14
    # stability polynomial of y' = y: coefficients 1, 1, 1/2, 1/6, 1/24
    s = len(A)
    coeffs = [1.0, b.sum()]
    Apow = np.eye(s)
    for k in range(2, 6):
        Apow = Apow @ a if k > 2 else a.copy()
        coeffs.append(b @ Apow @ np.ones(s))
    ref = [1, 1, 1 / 2, 1 / 6, 1 / 24]
    assert np.allclose(coeffs[:5], ref, rtol=0, atol=1e-14)
    assert abs(coeffs[5] - 1 / 120) > 1e-4  # 5 stages, 4th order: not 5th
    # the non-linear 4th-order conditions (Butcher trees of order 3 and 4)
    C = np.diag(c)
    one = np.ones(s)
    assert abs(b @ c ** 2 - 1 / 3) < 1e-14
    assert abs(b @ a @ c - 1 / 6) < 1e-14
    assert abs(b @ c ** 3 - 1 / 4) < 1e-14
    assert abs(b @ C @ a @ c - 1 / 8) < 1e-14
    assert abs(b @ a @ c ** 2 - 1 / 12) < 1e-14
    assert abs(b @ a @ a @ c - 1 / 24) < 1e-14
    assert A[0] == 0.0  # one state array suffices to restart a step
