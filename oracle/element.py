"""Hexahedral element operators by direct quadrature (oracle; test only).

Shape functions are the tensor products of eq. ProdTensorialHexaedro,
N_m(xi) = phi_p(xi_1) phi_q(xi_2) phi_r(xi_3), tabulated in full at all
Q^3 Gauss points (a dense Q^3 x n^3 matrix per derivative direction); there is
no sum factorisation.  Geometry: axis-aligned boxes, so the isoparametric map
of Sec. 3 (eq. interpolacao material coord) is affine with constant diagonal
Jacobian diag(h)/2.

Operators (vectorised over elements, arrays U[e, c, m]):

* internal force R = int P(F) : grad N  (second term of eq. material virtual
  work with S : dE = P : grad du);
* tangent action (dR/du) x = int grad N : A(F) : grad x  (Sec. 3,
  eq. effective stiffness 2);
* consistent mass action M x = int rho N N x  (first term of eq. material
  virtual work; global M of Sec. 4);
* dense element tangent and mass matrices for tiny meshes.
"""
import numpy as np

from . import material
from .quadrature import gauss_legendre, gauss_lobatto_legendre_rule


class RefElement:
    """rule "gauss": Q (default P + 2) Gauss-Legendre points per direction;
    rule "gll": the P + 1 Gauss-Lobatto-Legendre points (collocation
    integration at the nodes of the Lagrange basis, Sec. 2: with that basis
    the mass matrix is diagonal)."""

    def __init__(self, basis, h, Q=None, rule="gauss"):
        self.basis = basis
        self.P = basis.P
        self.n = basis.P + 1
        self.rule = rule
        if rule == "gll":
            self.Q = self.n
            xq, wq = gauss_lobatto_legendre_rule(self.P)
        else:
            self.Q = Q or (basis.P + 2)
            xq, wq = gauss_legendre(self.Q)
        self.xq, self.wq1 = xq, wq
        B, D = basis.tables(xq)
        self.B, self.D = B, D
        self.h = tuple(h)
        self.detJ = h[0] * h[1] * h[2] / 8.0
        k = np.kron
        self.N = k(B, k(B, B))
        self.dN = np.stack([
            k(B, k(B, D)) * (2.0 / h[0]),
            k(B, k(D, B)) * (2.0 / h[1]),
            k(D, k(B, B)) * (2.0 / h[2]),
        ])                                               # (3, Q^3, n^3)
        self.w = k(wq, k(wq, wq)) * self.detJ            # (Q^3,)

    # -- kinematics -------------------------------------------------------
    def grad(self, U):
        """G[e, q, c, d] = d u_c / d X_d at Gauss point q."""
        E = U.shape[0]
        Uf = U.reshape(E * 3, -1)
        G = np.stack([Uf @ self.dN[d].T for d in range(3)], axis=-1)   # (E*3, Q3, 3)
        return G.reshape(E, 3, -1, 3).transpose(0, 2, 1, 3)

    def values(self, U):
        E = U.shape[0]
        return (U.reshape(E * 3, -1) @ self.N.T).reshape(E, 3, -1).transpose(0, 2, 1)

    def divergence(self, Flux):
        """R[e, c, m] = sum_q sum_d w_q Flux[e, q, c, d] dN_d[q, m]."""
        E = Flux.shape[0]
        wF = Flux * self.w[None, :, None, None]
        out = np.zeros((E, 3, self.n ** 3))
        for d in range(3):
            Fd = wF[..., d].transpose(0, 2, 1).reshape(E * 3, -1)     # (E*3, Q3)
            out += (Fd @ self.dN[d]).reshape(E, 3, -1)
        return out

    def project(self, V):
        """R[e, c, m] = sum_q w_q V[e, q, c] N[q, m]."""
        E = V.shape[0]
        wV = (V * self.w[None, :, None]).transpose(0, 2, 1).reshape(E * 3, -1)
        return (wV @ self.N).reshape(E, 3, -1)

    # -- operators ----------------------------------------------------------
    def deformation(self, U):
        return np.eye(3)[None, None] + self.grad(U)

    def internal_force(self, U, mu, lam):
        F = self.deformation(U)
        if np.any(np.linalg.det(F) <= 0.0):
            raise FloatingPointError("non-positive J")
        return self.divergence(material.pk1(F, mu, lam))

    def energy(self, U, mu, lam):
        F = self.deformation(U)
        return np.einsum("eq,q->e", material.energy(F, mu, lam), self.w)

    def tangent_action(self, U, X, mu, lam):
        A = material.tangent(self.deformation(U), mu, lam)         # (E, Q3, 3,3,3,3)
        GX = self.grad(X)
        return self.divergence(np.einsum("eqiJkL,eqkL->eqiJ", A, GX))

    def mass_action(self, X, rho):
        return rho * self.project(self.values(X))

    def tangent_matrix(self, Ue, mu, lam):
        """Dense element tangent (3 n^3 x 3 n^3) of one element, index c*n^3+m."""
        A = material.tangent(self.deformation(Ue[None]), mu, lam)[0]   # (Q3,3,3,3,3)
        wA = A * self.w[:, None, None, None, None]
        n3, Q3 = self.n ** 3, self.Q ** 3
        dNt = self.dN.transpose(1, 0, 2)                          # (Q3, 3 D, n3)
        # T[q, c, d, k, m'] = sum_D wA[q, c, d, k, D] dN_D[q, m']
        T = np.matmul(wA.reshape(Q3, 27, 3), dNt).reshape(Q3, 3, 3, 3, n3)
        # K[c, m, k, m'] = sum_{q, d} dN_d[q, m] T[q, c, d, k, m']
        lhs = dNt.reshape(Q3 * 3, n3).T                           # (n3, (q, d))
        K = np.empty((3, n3, 3, n3))
        for c in range(3):
            K[c] = (lhs @ T[:, c].reshape(Q3 * 3, 3 * n3)).reshape(n3, 3, n3)
        return K.reshape(3 * n3, 3 * n3)

    def mass_matrix(self, rho):
        n3 = self.n ** 3
        Ms = rho * (self.N * self.w[:, None]).T @ self.N
        M = np.zeros((3, n3, 3, n3))
        for c in range(3):
            M[c, :, c, :] = Ms
        return M.reshape(3 * n3, 3 * n3)
