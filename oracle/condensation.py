"""Static condensation of the internal modes (oracle; test infrastructure only).

The paper solves its linear systems after a Schur complement on the element
internal modes (Sec. 4, the condensed system of the effective stiffness;
Sec. 5.1 states that the Schur complement is taken on the tangent matrix and
the residual).  With the lattice numbering, a lattice point is
element-interior when none of its three indices is a multiple of P: the
modes there (the internal modes of eq. BasePadrao1D, or the interior nodes
of the Lagrange basis) couple only within their element.  Splitting the
effective matrix A into skeleton (b) and interior (i) blocks,

    S = A_bb - A_bi A_ii^{-1} A_ib,   g = f_b - A_bi A_ii^{-1} f_i,
    S x_b = g,   x_i = A_ii^{-1} (f_i - A_ib x_b),

is the plain definition written out with sparse algebra; S is solved by the
same Jacobi-preconditioned CG (diagonal of S) as the uncondensed system.

Pins (tests/test_oracle_condensation.py): the condensed solution equals the
direct solution of the full system; the CG iteration counts per Newton
iteration reproduce the paper's static table (Sec. 5.1, Table
NH_average_IT_CGD) for the ST, SDME-M and SDME-H bases.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import solvers


def interior_mask(mesh):
    """True for DOFs of element-interior lattice points (all indices not multiples of P)."""
    P = mesh.P
    iz, iy, ix = np.meshgrid(np.arange(mesh.N[2]), np.arange(mesh.N[1]), np.arange(mesh.N[0]), indexing="ij")
    node = ((ix % P != 0) & (iy % P != 0) & (iz % P != 0)).ravel()
    return np.concatenate([node] * 3)


def condensed_solve(disc, u, f, b1=0.0, rtol=1e-12, maxit=100000):
    """Solve (b1 M + K_T(u)) x = f (Dirichlet-masked) through the Schur
    complement on the skeleton DOFs; returns (x, cg_iterations)."""
    A = disc.tangent_matrix(u, b1).tocsr()
    inner = interior_mask(disc.mesh)
    skel = ~inner
    Abb = A[skel][:, skel]
    Abi = A[skel][:, inner]
    Aib = A[inner][:, skel]
    lu = spla.splu(A[inner][:, inner].tocsc())
    f = np.where(disc.mask, 0.0, f)
    fb, fi = f[skel], f[inner]
    S = Abb - Abi @ sp.csr_matrix(lu.solve(Aib.toarray()))
    g = fb - Abi @ lu.solve(fi)
    d = S.diagonal()
    xb, its, _ = solvers.jacobi_pcg(lambda v: S @ v, g, d, rtol, maxit)
    x = np.zeros_like(f)
    x[skel] = xb
    x[inner] = lu.solve(fi - Aib @ xb)
    return x, its


def static_newton_condensed(disc, Pext, tol=1e-8, cg_rtol=1e-12, maxnewton=50):
    """Newton-Raphson for R(u) = P with condensed CG inner solves (Sec. 5.1)."""
    u = np.zeros(disc.mesh.ndof)
    psi0 = None
    its = []
    for k in range(maxnewton + 1):
        psi = Pext - disc.internal_force(u)
        psi[disc.mask] = 0.0
        nrm = np.linalg.norm(psi)
        psi0 = nrm if psi0 is None else psi0
        if nrm <= tol * max(psi0, np.linalg.norm(Pext)):
            return u, {"converged": True, "newton_iters": k, "cg_iters": its}
        if k == maxnewton:
            break
        du, n = condensed_solve(disc, u, psi, 0.0, cg_rtol)
        its.append(n)
        u = u + du
    return u, {"converged": False, "newton_iters": maxnewton, "cg_iters": its}
