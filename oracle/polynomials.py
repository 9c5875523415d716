"""Jacobi and Lagrange polynomials (oracle; test infrastructure only).

Sec. 2: the standard nodal basis is the Lagrange interpolant on the nodes
(eq. lagrangian, eq. shape_functions_lag); the standard modal basis uses the
Jacobi polynomials P_p^{alpha,beta} (eq. BasePadrao1D).
"""
import numpy as np


def jacobi(n, alpha, beta, x):
    """P_n^{alpha,beta}(x) by the textbook three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0
    p1 = 0.5 * ((alpha + beta + 2.0) * x + (alpha - beta))
    for k in range(1, n):
        s = 2.0 * k + alpha + beta
        c1 = 2.0 * (k + 1) * (k + alpha + beta + 1) * s
        c2 = (s + 1.0) * ((s + 2.0) * s * x + alpha * alpha - beta * beta)
        c3 = 2.0 * (k + alpha) * (k + beta) * (s + 2.0)
        p0, p1 = p1, (c2 * p1 - c3 * p0) / c1
    return p1


def jacobi_deriv(n, alpha, beta, x):
    """d/dx P_n^{alpha,beta}(x) = (n+alpha+beta+1)/2 P_{n-1}^{alpha+1,beta+1}."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    return 0.5 * (n + alpha + beta + 1.0) * jacobi(n - 1, alpha + 1.0, beta + 1.0, x)


def lagrange(nodes, a, x):
    """L_a(x) through ``nodes`` by the product formula of eq. lagrangian."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    for b, xb in enumerate(nodes):
        if b != a:
            out = out * (x - xb) / (nodes[a] - xb)
    return out


def lagrange_deriv(nodes, a, x):
    """d/dx L_a(x): derivative of the product formula, term by term."""
    x = np.asarray(x, dtype=np.float64)
    total = np.zeros_like(x)
    m = len(nodes)
    for k in range(m):
        if k == a:
            continue
        term = np.full_like(x, 1.0 / (nodes[a] - nodes[k]))
        for b in range(m):
            if b != a and b != k:
                term = term * (x - nodes[b]) / (nodes[a] - nodes[b])
        total = total + term
    return total
