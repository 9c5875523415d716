"""Global discretisation on a box mesh (oracle; test infrastructure only).

Gathers element coefficients from the global lattice, applies the dense
element operators of ``element.RefElement`` and sums element results back
(element-by-element assembly).  Also builds the global sparse tangent for
tiny meshes and the load vectors of eq. material virtual work (body force and
dead surface traction on box faces).
"""
import numpy as np
import scipy.sparse as sp

from .element import RefElement

_FACE_AXIS = {"xmin": (0, 0), "xmax": (0, 1), "ymin": (1, 0), "ymax": (1, 1),
              "zmin": (2, 0), "zmax": (2, 1)}


class Discretization:
    def __init__(self, mesh, basis, mu, lam, rho=1.0, Q=None, chunk=512, mass_rule="gauss"):
        """mass_rule "gll": the mass matrix (only) is integrated at the P + 1
        Gauss-Lobatto-Legendre points, which for the Lagrange basis on those
        points gives the diagonal (lumped) mass of the paper's explicit Lagrange
        runs; stiffness and loads keep the Gauss rule."""
        if basis.P != mesh.P:
            raise ValueError("basis order must match mesh order")
        self.mesh, self.basis = mesh, basis
        self.mu, self.lam, self.rho = float(mu), float(lam), float(rho)
        self.ref = RefElement(basis, mesh.h, Q)
        self.mref = RefElement(basis, mesh.h, rule="gll") if mass_rule == "gll" else self.ref
        self.edofs = mesh.element_dofs()
        self.mask = mesh.constrained()
        self.chunk = chunk

    # -- gather / scatter ------------------------------------------------
    def gather(self, x, elems=slice(None)):
        return x[self.edofs[elems]]

    def scatter(self, Ye, elems=slice(None)):
        return np.bincount(self.edofs[elems].ravel(), weights=Ye.ravel(),
                           minlength=self.mesh.ndof)

    def _chunks(self):
        E = self.mesh.nelem
        for s in range(0, E, self.chunk):
            yield slice(s, min(E, s + self.chunk))

    # -- global operators (unmasked) --------------------------------------
    def internal_force(self, u):
        out = np.zeros(self.mesh.ndof)
        for s in self._chunks():
            out += self.scatter(self.ref.internal_force(self.gather(u, s), self.mu, self.lam), s)
        return out

    def mass_apply(self, x):
        out = np.zeros(self.mesh.ndof)
        for s in self._chunks():
            out += self.scatter(self.mref.mass_action(self.gather(x, s), self.rho), s)
        return out

    def tangent_apply(self, u, x, b1=0.0):
        """(b1 M + K_T(u)) x, no Dirichlet treatment."""
        out = np.zeros(self.mesh.ndof)
        for s in self._chunks():
            Ue, Xe = self.gather(u, s), self.gather(x, s)
            Ye = self.ref.tangent_action(Ue, Xe, self.mu, self.lam)
            if b1 != 0.0:
                Ye = Ye + b1 * self.mref.mass_action(Xe, self.rho)
            out += self.scatter(Ye, s)
        return out

    def energy(self, u):
        return float(sum(self.ref.energy(self.gather(u, s), self.mu, self.lam).sum()
                         for s in self._chunks()))

    # -- Dirichlet-masked operators (rows and columns removed, unit diagonal)
    def effective_apply(self, u, x, b1=0.0):
        xm = np.where(self.mask, 0.0, x)
        y = self.tangent_apply(u, xm, b1)
        return np.where(self.mask, x, y)

    def diagonal(self, u, b1=0.0):
        """diag(b1 M + K_T(u)) with unit entries on constrained DOFs.

        The element diagonal is sum_q w_q sum_{d,d'} dN_d A_{c d c d'} dN_d'
        + b1 rho sum_q w_q N^2 at each (c, m); summed over elements."""
        from . import material
        ref = self.ref
        out = np.zeros(self.mesh.ndof)
        for s in self._chunks():
            F = ref.deformation(self.gather(u, s))
            A = material.tangent(F, self.mu, self.lam)
            E = F.shape[0]
            De = np.zeros((E, 3, ref.n ** 3))
            for c in range(3):
                for d in range(3):
                    for D in range(3):
                        tab = ref.dN[d] * ref.dN[D]                  # (Q3, n3)
                        De[:, c, :] += (A[:, :, c, d, c, D] * ref.w[None, :]) @ tab
            if b1 != 0.0:
                De += b1 * self.rho * (ref.w @ (ref.N * ref.N))[None, None, :]
            out += self.scatter(De, s)
        return np.where(self.mask, 1.0, out)

    def mass_diagonal(self):
        """diag(M): rho sum_q w_q N_m(q)^2 summed over elements."""
        De = self.rho * (self.mref.w @ (self.mref.N * self.mref.N))
        out = np.zeros(self.mesh.ndof)
        for s in self._chunks():
            E = s.stop - s.start
            out += self.scatter(np.broadcast_to(De, (E, 3, De.size)).copy(), s)
        return out

    def kinetic_energy(self, v):
        return 0.5 * float(v @ self.mass_apply(v))

    def tangent_matrix(self, u, b1=0.0, masked=True):
        """Global sparse b1 M + K_T(u) (tiny meshes)."""
        ref = self.ref
        Me = ref.mass_matrix(self.rho) if b1 != 0.0 else None
        rows, cols, vals = [], [], []
        U = self.gather(u)
        for e in range(self.mesh.nelem):
            Ke = ref.tangent_matrix(U[e], self.mu, self.lam)
            if Me is not None:
                Ke = Ke + b1 * Me
            idx = self.edofs[e].ravel()
            rows.append(np.repeat(idx, idx.size))
            cols.append(np.tile(idx, idx.size))
            vals.append(Ke.ravel())
        n = self.mesh.ndof
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(n, n))
        if masked:
            keep = sp.diags((~self.mask).astype(float))
            K = keep @ K @ keep + sp.diags(self.mask.astype(float))
        return K.tocsr()

    def mass_matrix(self):
        Me = self.mref.mass_matrix(self.rho)
        rows, cols, vals = [], [], []
        for e in range(self.mesh.nelem):
            idx = self.edofs[e].ravel()
            rows.append(np.repeat(idx, idx.size))
            cols.append(np.tile(idx, idx.size))
            vals.append(Me.ravel())
        n = self.mesh.ndof
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n, n))

    # -- geometry helpers ----------------------------------------------------
    def gauss_points(self, ref=None):
        """Physical coordinates X[e, q, 3] of the Gauss points of ``ref``."""
        ref = ref or self.ref
        Q = ref.Q
        xq = ref.xq
        k3, k2, k1 = np.meshgrid(np.arange(Q), np.arange(Q), np.arange(Q), indexing="ij")
        xi = np.stack([xq[k1.ravel()], xq[k2.ravel()], xq[k3.ravel()]], axis=-1)   # (Q3, 3)
        out = np.empty((self.mesh.nelem, Q ** 3, 3))
        for e in range(self.mesh.nelem):
            ec = self.mesh.elem_coords(e)
            for d in range(3):
                out[e, :, d] = (ec[d] + 0.5 * (1.0 + xi[:, d])) * self.mesh.h[d]
        return out

    # -- loads ---------------------------------------------------------------
    def body_load(self, bfunc, t=0.0):
        """f_(c,m) = int b_c(X, t) N_m dV (third term of eq. material virtual work)."""
        X = self.gauss_points()
        B = bfunc(X, t)                                                  # (E, Q3, 3)
        return self.scatter(self.ref.project(B))

    def traction_load(self, face, tfunc, t=0.0):
        """f_(c,m) = int_face t_c(X, t) N_m dA for a dead (reference) traction
        on one box face (fourth term of eq. material virtual work)."""
        mesh, basis = self.mesh, self.basis
        axis, side = _FACE_AXIS[face]
        tang = [d for d in range(3) if d != axis]
        Q = self.ref.Q
        xq, wq = self.ref.xq, self.ref.wq1                            # the element's own rule
        B, _ = basis.tables(xq)                                       # (Q, n)
        Bend, _ = basis.tables(np.array([-1.0 if side == 0 else 1.0]))  # (1, n)
        n = mesh.n
        out = np.zeros(mesh.ndof)
        jac = 0.25 * mesh.h[tang[0]] * mesh.h[tang[1]]
        for e in range(mesh.nelem):
            ec = mesh.elem_coords(e)
            if ec[axis] != (0 if side == 0 else mesh.ne[axis] - 1):
                continue
            # face Gauss points, a = first tangential axis (fast), b = second
            ka, kb = np.meshgrid(np.arange(Q), np.arange(Q), indexing="xy")
            ka, kb = ka.ravel(), kb.ravel()
            X = np.empty((Q * Q, 3))
            X[:, axis] = (ec[axis] + side) * mesh.h[axis]
            X[:, tang[0]] = (ec[tang[0]] + 0.5 * (1 + xq[ka])) * mesh.h[tang[0]]
            X[:, tang[1]] = (ec[tang[1]] + 0.5 * (1 + xq[kb])) * mesh.h[tang[1]]
            T = tfunc(X, t)                                             # (Q*Q, 3)
            w = wq[ka] * wq[kb] * jac
            # local 3D table of N_m on the face points
            tabs = [None, None, None]
            tabs[axis] = np.repeat(Bend, Q * Q, axis=0)
            tabs[tang[0]] = B[ka]
            tabs[tang[1]] = B[kb]
            Nf = np.einsum("sr,sq,sp->srqp", tabs[2], tabs[1], tabs[0]).reshape(Q * Q, n ** 3)
            fe = (T * w[:, None]).T @ Nf                                # (3, n3)
            idx = self.edofs[e]
            for c in range(3):
                np.add.at(out, idx[c], fe[c])
        return out

    # -- function-space helpers ----------------------------------------------
    def l2_error(self, u, exact, t=0.0, Qerr=None):
        """Per-component ||u_h - u||_{L2(Omega)} with a finer Gauss rule."""
        ref = RefElement(self.basis, self.mesh.h, Qerr or (self.mesh.P + 4))
        X = self.gauss_points(ref)
        uh = ref.values(self.gather(u))                                 # (E, Q3, 3)
        ue = exact(X, t)
        return np.sqrt(np.einsum("eqc,q->c", (uh - ue) ** 2, ref.w))

    def l2_project(self, func, t=0.0):
        """Coefficients of the L2 projection of ``func`` (direct solve)."""
        import scipy.sparse.linalg as spla
        rhs = self.scatter(self.ref.project(func(self.gauss_points(), t)))
        M = self.mass_matrix() / self.rho
        return spla.spsolve(M.tocsc(), rhs)


def elements_touching(mesh, dofs):
    """Indices of the elements whose coefficient set contains any of ``dofs``
    (used to evaluate sampled outputs of a large mesh element by element)."""
    P = mesh.P
    Nx, Ny, _ = mesh.N
    out = set()
    for g in np.atleast_1d(dofs):
        r = int(g) % mesh.Nn
        lat = (r % Nx, (r // Nx) % Ny, r // (Nx * Ny))
        cand = []
        for d in range(3):
            i = lat[d]
            es = {min(i // P, mesh.ne[d] - 1)}
            if i % P == 0 and i > 0:
                es.add(i // P - 1)
            cand.append(sorted(es))
        for ex in cand[0]:
            for ey in cand[1]:
                for ez in cand[2]:
                    out.add((ez * mesh.ne[1] + ey) * mesh.ne[0] + ex)
    return np.array(sorted(out), dtype=np.int64)
