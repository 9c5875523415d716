"""Plane-strain quadrilateral discretisation (oracle; test infrastructure only).

The 2D shape functions are the tensor products of eq. ProdTensorialQuadrado,
N_i(xi_1, xi_2) = phi_p(xi_1) phi_q(xi_2), on a structured rectangle of equal
quads (the 2D counterpart of ``hexmesh`` / ``assembly``).  The material is the
neo-Hookean law of Sec. 3 under plane strain: the 3D deformation gradient is
the in-plane F with F_33 = 1 (no out-of-plane displacement or dependence), and
the in-plane blocks of the 3D stress and tangent of ``material`` are used
(the definition of plane strain, no separate 2D formula).

Numbering: lattice Nx x Ny with Nd = nd P + 1; DOF (c, ix, iy) at
c Nn + iy Nx + ix (c = 0, 1; Nn = Nx Ny); element e = ey nx + ex; local mode
m = q n + p.  Dirichlet data are whole edges per component.

Pins (tests/test_oracle_quad.py): a 2D solution extruded through one layer
of hexahedra with every z-component clamped solves the 3D discrete problem
(exact relation between the 2D and 3D internal forces), finite differences
of the energy and of R, the small-strain limit, the affine patch test, and
the static fabricated field of Sec. 5.1 in plane strain (spectral
convergence in P, L2 rate P + 1 in h).
"""
import numpy as np
import scipy.sparse as sp

from . import material
from .quadrature import gauss_legendre

EDGES = ("xmin", "xmax", "ymin", "ymax")


def _embed(F2):
    """3x3 deformation gradients with the in-plane block F2 and F_33 = 1."""
    F3 = np.zeros(F2.shape[:-2] + (3, 3))
    F3[..., :2, :2] = F2
    F3[..., 2, 2] = 1.0
    return F3


class RectMesh:
    def __init__(self, nx, ny, P, lengths=(1.0, 1.0)):
        self.ne = (int(nx), int(ny))
        self.P = int(P)
        self.n = self.P + 1
        self.lengths = tuple(float(v) for v in lengths)
        self.h = tuple(self.lengths[d] / self.ne[d] for d in range(2))
        self.N = tuple(self.ne[d] * self.P + 1 for d in range(2))
        self.Nn = self.N[0] * self.N[1]
        self.ndof = 2 * self.Nn
        self.nelem = self.ne[0] * self.ne[1]
        self.dirichlet = {f: () for f in EDGES}

    def elem_coords(self, e):
        return e % self.ne[0], e // self.ne[0]

    def element_dofs(self):
        """Array (nelem, 2, n^2) of global DOF indices per element."""
        n, P = self.n, self.P
        q, p = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        p, q = p.ravel(), q.ravel()
        out = np.empty((self.nelem, 2, n * n), dtype=np.int64)
        for e in range(self.nelem):
            ex, ey = self.elem_coords(e)
            nodes = (ey * P + q) * self.N[0] + ex * P + p
            for c in range(2):
                out[e, c] = c * self.Nn + nodes
        return out

    def clamp(self, edge, comps=(0, 1)):
        self.dirichlet[edge] = tuple(sorted(set(self.dirichlet[edge]) | set(comps)))
        return self

    def constrained(self):
        Nx, Ny = self.N
        iy, ix = np.meshgrid(np.arange(Ny), np.arange(Nx), indexing="ij")
        ix, iy = ix.ravel(), iy.ravel()
        on = {"xmin": ix == 0, "xmax": ix == Nx - 1, "ymin": iy == 0, "ymax": iy == Ny - 1}
        mask = np.zeros(self.ndof, dtype=bool)
        for f, comps in self.dirichlet.items():
            for c in comps:
                mask[c * self.Nn:(c + 1) * self.Nn] |= on[f]
        return mask


class RefQuad:
    """Dense 2D element operators by direct quadrature (Q x Q Gauss points)."""

    def __init__(self, basis, h, Q=None):
        self.basis = basis
        self.P = basis.P
        self.n = basis.P + 1
        self.Q = Q or (basis.P + 2)
        xq, wq = gauss_legendre(self.Q)
        self.xq, self.wq1 = xq, wq
        B, D = basis.tables(xq)
        self.h = tuple(h)
        self.detJ = h[0] * h[1] / 4.0
        k = np.kron
        self.N = k(B, B)                                                 # (Q2, n2): index qy*Q+qx, q*n+p
        self.dN = np.stack([k(B, D) * (2.0 / h[0]), k(D, B) * (2.0 / h[1])])
        self.w = k(wq, wq) * self.detJ

    def grad(self, U):
        E = U.shape[0]
        Uf = U.reshape(E * 2, -1)
        G = np.stack([Uf @ self.dN[d].T for d in range(2)], axis=-1)    # (E*2, Q2, 2)
        return G.reshape(E, 2, -1, 2).transpose(0, 2, 1, 3)

    def deformation(self, U):
        return np.eye(2)[None, None] + self.grad(U)

    def divergence(self, Flux):
        E = Flux.shape[0]
        wF = Flux * self.w[None, :, None, None]
        out = np.zeros((E, 2, self.n ** 2))
        for d in range(2):
            Fd = wF[..., d].transpose(0, 2, 1).reshape(E * 2, -1)
            out += (Fd @ self.dN[d]).reshape(E, 2, -1)
        return out

    def values(self, U):
        E = U.shape[0]
        return (U.reshape(E * 2, -1) @ self.N.T).reshape(E, 2, -1).transpose(0, 2, 1)

    def project(self, V):
        E = V.shape[0]
        wV = (V * self.w[None, :, None]).transpose(0, 2, 1).reshape(E * 2, -1)
        return (wV @ self.N).reshape(E, 2, -1)

    def internal_force(self, U, mu, lam):
        F = self.deformation(U)
        if np.any(np.linalg.det(F) <= 0.0):
            raise FloatingPointError("non-positive J")
        return self.divergence(material.pk1(_embed(F), mu, lam)[..., :2, :2])

    def energy(self, U, mu, lam):
        return np.einsum("eq,q->e", material.energy(_embed(self.deformation(U)), mu, lam), self.w)

    def tangent_action(self, U, X, mu, lam):
        A = material.tangent(_embed(self.deformation(U)), mu, lam)[..., :2, :2, :2, :2]
        return self.divergence(np.einsum("eqiJkL,eqkL->eqiJ", A, self.grad(X)))

    def mass_action(self, X, rho):
        return rho * self.project(self.values(X))

    def tangent_matrix(self, Ue, mu, lam):
        """Dense element tangent (2 n^2 x 2 n^2), index c*n^2+m, by columns."""
        n2 = self.n ** 2
        K = np.empty((2 * n2, 2 * n2))
        for j in range(2 * n2):
            X = np.zeros((1, 2, n2))
            X.reshape(-1)[j] = 1.0
            K[:, j] = self.tangent_action(Ue[None], X, mu, lam).reshape(-1)
        return K

    def mass_matrix(self, rho):
        n2 = self.n ** 2
        Ms = rho * (self.N * self.w[:, None]).T @ self.N
        M = np.zeros((2, n2, 2, n2))
        for c in range(2):
            M[c, :, c, :] = Ms
        return M.reshape(2 * n2, 2 * n2)


class Discretization2D:
    def __init__(self, mesh, basis, mu, lam, rho=1.0, Q=None):
        if basis.P != mesh.P:
            raise ValueError("basis order must match mesh order")
        self.mesh, self.basis = mesh, basis
        self.mu, self.lam, self.rho = float(mu), float(lam), float(rho)
        self.ref = RefQuad(basis, mesh.h, Q)
        self.edofs = mesh.element_dofs()
        self.mask = mesh.constrained()

    def gather(self, x):
        return x[self.edofs]

    def scatter(self, Ye):
        out = np.zeros(self.mesh.ndof)
        np.add.at(out, self.edofs.reshape(-1), Ye.reshape(-1))
        return out

    def internal_force(self, u):
        return self.scatter(self.ref.internal_force(self.gather(u), self.mu, self.lam))

    def energy(self, u):
        return float(self.ref.energy(self.gather(u), self.mu, self.lam).sum())

    def mass_apply(self, x):
        return self.scatter(self.ref.mass_action(self.gather(x), self.rho))

    def kinetic_energy(self, v):
        return 0.5 * float(v @ self.mass_apply(v))

    def tangent_apply(self, u, x, b1=0.0):
        """(b1 M + K_T(u)) x, no Dirichlet treatment."""
        Ue, Xe = self.gather(u), self.gather(x)
        Ye = self.ref.tangent_action(Ue, Xe, self.mu, self.lam)
        if b1 != 0.0:
            Ye = Ye + b1 * self.ref.mass_action(Xe, self.rho)
        return self.scatter(Ye)

    def effective_apply(self, u, x, b1=0.0):
        xm = np.where(self.mask, 0.0, x)
        y = self.tangent_apply(u, xm, b1)
        return np.where(self.mask, x, y)

    def tangent_matrix(self, u, b1=0.0, masked=True):
        Me = self.ref.mass_matrix(self.rho) if b1 != 0.0 else None
        rows, cols, vals = [], [], []
        U = self.gather(u)
        for e in range(self.mesh.nelem):
            Ke = self.ref.tangent_matrix(U[e], self.mu, self.lam)
            if Me is not None:
                Ke = Ke + b1 * Me
            idx = self.edofs[e].ravel()
            rows.append(np.repeat(idx, idx.size))
            cols.append(np.tile(idx, idx.size))
            vals.append(Ke.ravel())
        n = self.mesh.ndof
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
        if masked:
            keep = sp.diags((~self.mask).astype(float))
            K = keep @ K @ keep + sp.diags(self.mask.astype(float))
        return K.tocsr()

    def diagonal(self, u, b1=0.0):
        """diag(b1 M + K_T(u)) with unit entries on constrained DOFs."""
        return np.where(self.mask, 1.0, self.tangent_matrix(u, b1, masked=False).diagonal())

    def mass_matrix(self):
        Me = self.ref.mass_matrix(self.rho)
        rows, cols, vals = [], [], []
        for e in range(self.mesh.nelem):
            idx = self.edofs[e].ravel()
            rows.append(np.repeat(idx, idx.size))
            cols.append(np.tile(idx, idx.size))
            vals.append(Me.ravel())
        n = self.mesh.ndof
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))

    def gauss_points(self, ref=None):
        """Physical coordinates X[e, q, 2] of the Gauss points of ``ref``
        (q = qy Q + qx, the order of ``RefQuad``)."""
        ref = ref or self.ref
        Q, xq = ref.Q, ref.xq
        ky, kx = np.meshgrid(np.arange(Q), np.arange(Q), indexing="ij")
        xi = np.stack([xq[kx.ravel()], xq[ky.ravel()]], axis=-1)           # (Q2, 2)
        out = np.empty((self.mesh.nelem, Q * Q, 2))
        for e in range(self.mesh.nelem):
            ec = self.mesh.elem_coords(e)
            for d in range(2):
                out[e, :, d] = (ec[d] + 0.5 * (1.0 + xi[:, d])) * self.mesh.h[d]
        return out

    def body_load(self, bfunc, t=0.0):
        """f = int b(X, t) N dA per unit thickness (third term of eq. material
        virtual work in plane strain); bfunc maps X[..., 2] to b[..., 2]."""
        return self.scatter(self.ref.project(bfunc(self.gauss_points(), t)))

    def traction_field_load(self, edge, tfunc, t=0.0):
        """f = int_edge t(X, t) N ds for a dead traction that may vary along
        the edge (fourth term of eq. material virtual work, per unit thickness);
        tfunc maps X[..., 2] to t[..., 2]."""
        mesh, basis = self.mesh, self.basis
        axis = 0 if edge in ("xmin", "xmax") else 1
        side = 1 if edge in ("xmax", "ymax") else 0
        tang = 1 - axis
        xq, wq = self.ref.xq, self.ref.wq1
        B, _ = basis.tables(xq)                                         # (Q, n) along the edge
        Bend, _ = basis.tables(np.array([1.0 if side else -1.0]))       # (1, n) across it
        n = mesh.n
        jac = 0.5 * mesh.h[tang]
        Ye = np.zeros((mesh.nelem, 2, n * n))
        for e in range(mesh.nelem):
            ec = mesh.elem_coords(e)
            if ec[axis] != (mesh.ne[axis] - 1 if side else 0):
                continue
            X = np.empty((xq.size, 2))
            X[:, axis] = (ec[axis] + side) * mesh.h[axis]
            X[:, tang] = (ec[tang] + 0.5 * (1.0 + xq)) * mesh.h[tang]
            T = tfunc(X, t)                                             # (Q, 2)
            along = (wq[:, None] * B).T @ T * jac                       # (n, 2): int t_c phi_a ds
            for a in range(n):
                for b in range(n):
                    # local mode m = q n + p with p along x, q along y
                    p_, q_ = (b, a) if axis == 0 else (a, b)
                    Ye[e, :, q_ * n + p_] += along[a] * Bend[0, b]
        return self.scatter(Ye)

    def l2_error(self, u, exact, t=0.0, Qerr=None):
        """Per-component ||u_h - u||_{L2} with a finer Gauss rule."""
        ref = RefQuad(self.basis, self.mesh.h, Qerr or (self.mesh.P + 4))
        X = self.gauss_points(ref)
        uh = ref.values(self.gather(u))                                 # (E, Q2, 2)
        ue = exact(X, t)
        return np.sqrt(np.einsum("eqc,q->c", (uh - ue) ** 2, ref.w))

    def traction_load(self, edge, t):
        """f = int_edge t N ds for a uniform dead traction t (2-vector) on one edge."""
        mesh, basis = self.mesh, self.basis
        axis = 0 if edge in ("xmin", "xmax") else 1
        side = 1 if edge in ("xmax", "ymax") else 0
        tang = 1 - axis
        xq, wq = gauss_legendre(self.ref.Q)
        B, _ = basis.tables(xq)
        I = wq @ B                                                      # int phi_j
        out = np.zeros(mesh.ndof)
        fixed = side * (mesh.N[axis] - 1)
        jac = 0.5 * mesh.h[tang]
        for et in range(mesh.ne[tang]):
            for a in range(mesh.n):
                idx = [0, 0]
                idx[axis] = fixed
                idx[tang] = et * mesh.P + a
                node = idx[1] * mesh.N[0] + idx[0]
                for c in range(2):
                    out[c * mesh.Nn + node] += t[c] * jac * I[a]
        return out
