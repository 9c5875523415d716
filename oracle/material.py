"""Compressible neo-Hookean material (oracle; test infrastructure only).

Sec. 3 of the paper: strain energy (eq. hyperelastic strain energy)

    Psi = mu/2 (tr C - 3) - mu ln J + lambda/2 (ln J)^2,

and second Piola-Kirchhoff stress (eq. second Piolla_Kirchhoff relation)

    S = mu (I - C^{-1}) + lambda ln J C^{-1},    C = F^T F,  J = det F.

The virtual work of eq. material virtual work is S : delta E, which equals
(F S) : grad(delta u); the oracle therefore assembles with the first
Piola-Kirchhoff stress P = F S.  The consistent tangent dP/dF is written from
the material elasticity tensor of the same energy (Bonet & Wood's form):

    C_IJKL = lambda Cinv_IJ Cinv_KL + (mu - lambda ln J)(Cinv_IK Cinv_JL + Cinv_IL Cinv_JK)
    A_iJkL = delta_ik S_JL + F_iI F_kK C_IJKL.

All functions are vectorised over leading axes of F (shape (..., 3, 3)).
"""
import numpy as np


def lame(E, nu):
    """Lame parameters (mu, lambda) from Young's modulus and Poisson's ratio."""
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def energy(F, mu, lam):
    """Psi(F) of eq. hyperelastic strain energy."""
    C = np.einsum("...ki,...kj->...ij", F, F)
    J = np.linalg.det(F)
    lnJ = np.log(J)
    trC = np.trace(C, axis1=-2, axis2=-1)
    return 0.5 * mu * (trC - 3.0) - mu * lnJ + 0.5 * lam * lnJ ** 2


def pk2(F, mu, lam):
    """S(F) of eq. second Piolla_Kirchhoff relation."""
    C = np.einsum("...ki,...kj->...ij", F, F)
    Ci = np.linalg.inv(C)
    J = np.linalg.det(F)
    I = np.broadcast_to(np.eye(3), C.shape)
    return mu * (I - Ci) + lam * np.log(J)[..., None, None] * Ci


def pk1(F, mu, lam):
    """First Piola-Kirchhoff stress P = F S."""
    return np.einsum("...ij,...jk->...ik", F, pk2(F, mu, lam))


def tangent(F, mu, lam):
    """A[..., i, J, k, L] = dP_iJ / dF_kL (see module docstring)."""
    C = np.einsum("...ki,...kj->...ij", F, F)
    Ci = np.linalg.inv(C)
    J = np.linalg.det(F)
    lnJ = np.log(J)[..., None, None, None, None]
    S = pk2(F, mu, lam)
    CC = (lam * np.einsum("...IJ,...KL->...IJKL", Ci, Ci)
          + (mu - lam * lnJ) * (np.einsum("...IK,...JL->...IJKL", Ci, Ci)
                                + np.einsum("...IL,...JK->...IJKL", Ci, Ci)))
    geo = np.einsum("ik,...JL->...iJkL", np.eye(3), S)
    mat = np.einsum("...iI,...kK,...IJKL->...iJkL", F, F, CC)
    return geo + mat


def linear_elastic_tangent(mu, lam):
    """Small-strain elasticity tensor lambda d_ij d_kl + mu (d_ik d_jl + d_il d_jk)."""
    d = np.eye(3)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))
