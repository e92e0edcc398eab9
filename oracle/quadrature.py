"""Gauss-Legendre and Gauss-Lobatto rules on [0, 1] (oracle; test infrastructure only).

The paper integrates its element forms by quadrature (Sec. 2.1) without naming a
rule. Reading used throughout: (k+2)-point Gauss-Legendre per direction for RT_k.
Nodes come from Newton's method on Legendre polynomials evaluated by the
three-term recurrence (Abramowitz & Stegun 8.5.3, 25.4.29 and 25.4.32).
"""
from __future__ import annotations

import numpy as np


def legendre(n: int, x):
    """P_n(x) and P_n'(x) by (m+1) P_{m+1} = (2m+1) x P_m - m P_{m-1}."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for m in range(1, n):
        p0, p1 = p1, ((2 * m + 1) * x * p1 - m * p0) / (m + 1)
    # P_n' = n (x P_n - P_{n-1}) / (x^2 - 1) away from +-1; P_n'(+-1) = (+-1)^(n+1) n(n+1)/2
    end = np.abs(x) == 1.0
    den = np.where(end, 1.0, x * x - 1.0)
    dp = np.where(end, np.sign(x) ** (n + 1) * 0.5 * n * (n + 1), n * (x * p1 - p0) / den)
    return p1, dp


def gauss_legendre(q: int):
    """q-point Gauss-Legendre rule on [0,1]: nodes ascending, weights summing to 1."""
    if q < 1:
        raise ValueError("q >= 1")
    i = np.arange(1, q + 1)
    x = -np.cos(np.pi * (i - 0.25) / (q + 0.5))       # ascending initial guesses
    for _ in range(100):
        p, dp = legendre(q, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    _, dp = legendre(q, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_lobatto(q: int):
    """q-point Gauss-Lobatto rule on [0,1] (endpoints included), q >= 2.

    Interior nodes are the roots of P_{q-1}'; Newton uses P'' from the Legendre
    equation (1-x^2) P'' = 2x P' - n(n+1) P. Weights 2 / (n(n+1) P_n(x)^2), n = q-1.
    """
    if q < 2:
        raise ValueError("q >= 2")
    n = q - 1
    x = -np.cos(np.pi * np.arange(q) / n)             # Chebyshev-Lobatto start, ascending
    xi = x[1:-1].copy()
    for _ in range(100):
        if xi.size == 0:
            break
        p, dp = legendre(n, xi)
        d2p = (2.0 * xi * dp - n * (n + 1) * p) / (1.0 - xi * xi)
        dx = dp / d2p
        xi = xi - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    x = np.concatenate([[-1.0], xi, [1.0]])
    p, _ = legendre(n, x)
    w = 2.0 / (n * (n + 1) * p * p)
    return 0.5 * (x + 1.0), 0.5 * w
