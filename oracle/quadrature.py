"""1D quadrature rules (oracle; test infrastructure only).

Sec. 2 of the paper integrates the 1D mass and stiffness matrices (eqs.
Matrizesmassa, Matrizesrigidez) and places Lagrange nodes on
Gauss-Lobatto-Legendre points (text after eq. lagrangian).  The volume rule is
not stated; the reading used throughout is Q = P + 2 Gauss-Legendre points per
direction.

Both rules are computed by the Golub-Welsch method: the nodes are the
eigenvalues of the symmetric tridiagonal Jacobi matrix of the orthogonal
polynomial family and the weights come from the first eigenvector components.
"""
import numpy as np


def _jacobi_matrix(m, alpha, beta):
    """Symmetric tridiagonal recurrence matrix of the monic Jacobi family
    P_k^{alpha,beta}, size m x m (textbook three-term recurrence)."""
    a = np.zeros(m)
    b = np.zeros(max(m - 1, 0))
    for k in range(m):
        s = 2.0 * k + alpha + beta
        if abs(s * (s + 2.0)) > 0.0:
            a[k] = (beta * beta - alpha * alpha) / (s * (s + 2.0))
        else:
            a[k] = (beta - alpha) / (alpha + beta + 2.0)
    for k in range(1, m):
        s = 2.0 * k + alpha + beta
        num = 4.0 * k * (k + alpha) * (k + beta) * (k + alpha + beta)
        den = s * s * (s + 1.0) * (s - 1.0)
        b[k - 1] = np.sqrt(num / den)
    return np.diag(a) + np.diag(b, 1) + np.diag(b, -1)


def gauss_jacobi(m, alpha=0.0, beta=0.0):
    """m-point Gauss-Jacobi rule for weight (1-x)^alpha (1+x)^beta on [-1, 1].

    Returns (nodes ascending, weights).  Exact for polynomials of degree
    2m - 1 times the weight.
    """
    if m < 1:
        raise ValueError("need at least one point")
    J = _jacobi_matrix(m, alpha, beta)
    lam, V = np.linalg.eigh(J)
    # integral of the weight function over [-1, 1]
    from math import lgamma, exp, log
    mu0 = exp((alpha + beta + 1.0) * log(2.0) + lgamma(alpha + 1.0)
              + lgamma(beta + 1.0) - lgamma(alpha + beta + 2.0))
    w = mu0 * V[0, :] ** 2
    order = np.argsort(lam)
    return lam[order], w[order]


def gauss_legendre(m):
    """m-point Gauss-Legendre rule (Gauss-Jacobi with alpha = beta = 0)."""
    return gauss_jacobi(m, 0.0, 0.0)


def gauss_lobatto_legendre(P):
    """The P + 1 Gauss-Lobatto-Legendre points on [-1, 1] (Sec. 2).

    The interior points are the roots of P'_P, which are the Gauss points of
    the Jacobi weight (1-x)(1+x); the end points are -1 and +1.
    """
    if P < 1:
        raise ValueError("P must be >= 1")
    if P == 1:
        return np.array([-1.0, 1.0])
    inner, _ = gauss_jacobi(P - 1, 1.0, 1.0)
    return np.concatenate(([-1.0], inner, [1.0]))


def gauss_lobatto_legendre_rule(P):
    """P + 1 point Gauss-Lobatto-Legendre rule (nodes, weights): the nodes of
    ``gauss_lobatto_legendre`` with the textbook weights
    w_i = 2 / (P (P + 1) L_P(x_i)^2), L_P the Legendre polynomial (three-term
    recurrence).  Exact for polynomials of degree 2P - 1."""
    x = gauss_lobatto_legendre(P)
    L0, L1 = np.ones_like(x), x.copy()
    for k in range(1, P):
        L0, L1 = L1, ((2 * k + 1) * x * L1 - k * L0) / (k + 1)
    LP = L1 if P >= 1 else L0
    return x, 2.0 / (P * (P + 1) * LP * LP)
