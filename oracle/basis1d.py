"""1D expansion bases: standard nodal/modal, SD internal modes, ME boundary modes.

Oracle; test infrastructure only.  Follows Sec. 2 of the paper in its own
order:

1. standard bases psi_p (eq. shape_functions_lag for Lagrange on GLL nodes,
   eq. BasePadrao1D for the Jacobi modal basis, alpha = beta = 1 by default);
2. 1D mass and stiffness matrices (eqs. Matrizesmassa, Matrizesrigidez),
   integrated exactly with enough Gauss-Legendre points;
3. vertex / internal partition (eq. BlocosMassa);
4. simultaneous diagonalisation of the internal block (eqs. Diagonalizacao1,
   MatrizInterna, diagMassa, L, diagL, Y): eigen-decompose M_ii, form L, eigen-
   decompose L, and take Y = (X Lambda_M^{-1/2} Z Lambda_S^{-k/2})^T;
5. minimum-energy vertex modes (eq. ExtensaoMEmassa) with alpha = G_vi G_ii^{-1}
   for G = M (eq. alphaMassa, SDME-M), K (eq. alphaRigidez, SDME-K) or
   K + lambda M (eqs. EffectiveStiffness_lambda, alphaKN, SDME-H).

Readings where the paper is silent:

* Eigenvectors are fixed up to sign only.  Each new internal function is given
  the sign that makes its derivative at xi = -1 positive, and the internal
  functions are ordered by ascending eigenvalue of L.  This makes the basis
  independent of the eigensolver and of the standard basis it starts from.
* The ME step uses the original standard internal functions psi_j^i, as eq.
  ExtensaoMEmassa writes it; the result is the same function when the
  SD-transformed ones are used (checked in the tests).

Ordering.  Functions are held in the paper's order (0: vertex at -1, 1: vertex
at +1, 2..P: internal).  ``lattice_order`` maps them to the order used on the
global lattice: [vertex -1, internal 2..P, vertex +1].
"""
import numpy as np

from .polynomials import jacobi, jacobi_deriv, lagrange, lagrange_deriv
from .quadrature import gauss_legendre, gauss_lobatto_legendre

KINDS = ("nodal", "modal", "sdme_m", "sdme_k", "sdme_h")


class StandardBasis:
    """Standard (ST) 1D basis of order P in the paper's order."""

    def __init__(self, P, family="modal", alpha=1.0, beta=1.0):
        if P < 1:
            raise ValueError("P >= 1")
        if family not in ("modal", "nodal"):
            raise ValueError(family)
        self.P = P
        self.family = family
        self.alpha = alpha
        self.beta = beta
        if family == "nodal":
            self.nodes = gauss_lobatto_legendre(P)
            # paper order: L_0, L_P, then the body nodes 1..P-1
            self._lag_index = [0, P] + list(range(1, P))

    def eval(self, x):
        """Return (values, derivatives), each of shape (P+1, len(x))."""
        x = np.atleast_1d(np.asarray(x, dtype=np.float64))
        n = self.P + 1
        V = np.zeros((n, x.size))
        D = np.zeros((n, x.size))
        if self.family == "modal":
            # eq. BasePadrao1D
            V[0] = 0.5 * (1.0 - x)
            D[0] = -0.5
            V[1] = 0.5 * (1.0 + x)
            D[1] = 0.5
            bub = 0.25 * (1.0 - x) * (1.0 + x)
            dbub = -0.5 * x
            for p in range(2, n):
                J = jacobi(p - 2, self.alpha, self.beta, x)
                dJ = jacobi_deriv(p - 2, self.alpha, self.beta, x)
                V[p] = bub * J
                D[p] = dbub * J + bub * dJ
        else:
            # eqs. lagrangian, shape_functions_lag
            for p, a in enumerate(self._lag_index):
                V[p] = lagrange(self.nodes, a, x)
                D[p] = lagrange_deriv(self.nodes, a, x)
        return V, D


def matrices_1d(std, nquad=None):
    """1D mass and stiffness matrices of eqs. Matrizesmassa / Matrizesrigidez.

    Integrated with ``nquad`` Gauss-Legendre points (default P + 2, exact for
    the degree-2P integrands).
    """
    P = std.P
    nq = nquad or (P + 2)
    xq, wq = gauss_legendre(nq)
    V, D = std.eval(xq)
    M = (V * wq) @ V.T
    K = (D * wq) @ D.T
    return M, K


class Basis1D:
    """A 1D basis phi = T psi built from a standard basis psi (paper order)."""

    def __init__(self, P, kind, k=0.5, lam=100.0, start=None, alpha=1.0, beta=1.0):
        if kind not in KINDS:
            raise ValueError(kind)
        self.P = P
        self.kind = kind
        self.k = k
        self.lam = lam
        if start is None:
            start = "nodal" if kind == "nodal" else "modal"
        self.std = StandardBasis(P, start, alpha, beta)
        n = P + 1
        M, K = matrices_1d(self.std)
        self.M_std, self.K_std = M, K
        T = np.eye(n)
        self.lambda_S = None
        if kind.startswith("sdme") and P >= 2:
            Y, lamS = simultaneous_diagonalisation(M, K, k)
            # sign: derivative of each new internal function at xi = -1 > 0
            _, Dm1 = self.std.eval(np.array([-1.0]))
            d = Y @ Dm1[2:, 0]
            Y = Y * np.where(d < 0.0, -1.0, 1.0)[:, None]
            T[2:, 2:] = Y
            self.lambda_S = lamS
            G = {"sdme_m": M, "sdme_k": K, "sdme_h": K + lam * M}[kind]
            alpha_me = minimum_energy_alpha(G)
            T[0:2, 2:] = -alpha_me
            self.alpha_me = alpha_me
        self.T = T

    # -- evaluation -------------------------------------------------------
    def eval(self, x):
        """(values, derivatives) of the final functions, paper order."""
        V, D = self.std.eval(x)
        return self.T @ V, self.T @ D

    def matrices(self):
        """Mass and stiffness of the final basis, T M T^T and T K T^T."""
        return self.T @ self.M_std @ self.T.T, self.T @ self.K_std @ self.T.T

    @property
    def lattice_order(self):
        return [0] + list(range(2, self.P + 1)) + [1]

    def tables(self, xq):
        """B[q, j] = phi_j(x_q), D[q, j] = phi_j'(x_q), lattice order."""
        V, D = self.eval(xq)
        o = self.lattice_order
        return V[o].T.copy(), D[o].T.copy()


def simultaneous_diagonalisation(M, K, k):
    """Y of eq. Y for the internal blocks of M and K (paper order input).

    eq. diagMassa: X^T M_ii X = Lambda_M;  eq. L: L = (X Lambda_M^{-1/2})^T K_ii
    (X Lambda_M^{-1/2});  eq. diagL: Z^T L Z = Lambda_S;  eq. Y:
    Y = (X Lambda_M^{-1/2} Z Lambda_S^{-k/2})^T.  Returns (Y, Lambda_S) with
    Lambda_S ascending.
    """
    Mii = M[2:, 2:]
    Kii = K[2:, 2:]
    lamM, X = np.linalg.eigh(Mii)
    A = X * (lamM ** -0.5)[None, :]
    L = A.T @ Kii @ A
    L = 0.5 * (L + L.T)
    lamS, Z = np.linalg.eigh(L)
    Y = (A @ Z * (lamS ** (-0.5 * k))[None, :]).T
    return Y, lamS


def minimum_energy_alpha(G):
    """alpha = G_vi G_ii^{-1} (eqs. alphaMassa, alphaRigidez, alphaKN)."""
    Gvi = G[0:2, 2:]
    Gii = G[2:, 2:]
    return np.linalg.solve(Gii.T, Gvi.T).T
