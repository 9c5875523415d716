"""Structured box meshes of tensor-product hexahedra (oracle; test only).

The domain is [0, Lx] x [0, Ly] x [0, Lz] cut into nx x ny x nz equal hexes
of order P.  All elements share one orientation, so the 1D modes on a shared
edge or face are seen identically from both sides and C0 continuity needs no
sign flips (the conformity statement after eq. ProdTensorialHexaedro).

Global numbering: the (P+1)^3 coefficients of each element sit on a global
lattice of Nx x Ny x Nz points, Nd = nd P + 1.  The lattice index of element
(ex, ey, ez) and local mode (p, q, r) (lattice order, see ``basis1d``) is
(ex P + p, ey P + q, ez P + r).  DOF (c, ix, iy, iz) has index
c Nn + (iz Ny + iy) Nx + ix with Nn = Nx Ny Nz (component-major).
Element index e = (ez ny + ey) nx + ex; local mode index m = (r n + q) n + p.
"""
import numpy as np

FACES = ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")


class BoxMesh:
    def __init__(self, nx, ny, nz, P, lengths=(1.0, 1.0, 1.0)):
        self.ne = (int(nx), int(ny), int(nz))
        self.P = int(P)
        self.n = self.P + 1
        self.lengths = tuple(float(v) for v in lengths)
        self.h = tuple(self.lengths[d] / self.ne[d] for d in range(3))
        self.N = tuple(self.ne[d] * self.P + 1 for d in range(3))
        self.Nn = self.N[0] * self.N[1] * self.N[2]
        self.ndof = 3 * self.Nn
        self.nelem = self.ne[0] * self.ne[1] * self.ne[2]
        self.dirichlet = {f: () for f in FACES}

    # -- numbering ----------------------------------------------------------
    def node_index(self, ix, iy, iz):
        Nx, Ny, _ = self.N
        return (iz * Ny + iy) * Nx + ix

    def dof(self, c, ix, iy, iz):
        return c * self.Nn + self.node_index(ix, iy, iz)

    def elem_coords(self, e):
        nx, ny, _ = self.ne
        return e % nx, (e // nx) % ny, e // (nx * ny)

    def element_dofs(self):
        """Array (nelem, 3, n^3) of global DOF indices per element."""
        n, P = self.n, self.P
        r, q, p = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        p, q, r = p.ravel(), q.ravel(), r.ravel()          # m = (r n + q) n + p
        out = np.empty((self.nelem, 3, n ** 3), dtype=np.int64)
        for e in range(self.nelem):
            ex, ey, ez = self.elem_coords(e)
            nodes = self.node_index(ex * P + p, ey * P + q, ez * P + r)
            for c in range(3):
                out[e, c] = c * self.Nn + nodes
        return out

    # -- Dirichlet ------------------------------------------------------------
    def clamp(self, face, comps=(0, 1, 2)):
        self.dirichlet[face] = tuple(sorted(set(self.dirichlet[face]) | set(comps)))
        return self

    def constrained(self):
        """Boolean mask (ndof,) of DOFs on clamped faces.

        A coefficient lies on face x = 0 exactly when its lattice index ix = 0:
        every other 1D function vanishes at xi = -1 (vertex and ME modes keep
        phi_k(+-1) = delta), so the trace on the face involves only those.
        """
        Nx, Ny, Nz = self.N
        iz, iy, ix = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
        ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
        on = {"xmin": ix == 0, "xmax": ix == Nx - 1, "ymin": iy == 0,
              "ymax": iy == Ny - 1, "zmin": iz == 0, "zmax": iz == Nz - 1}
        mask = np.zeros(self.ndof, dtype=bool)
        for f, comps in self.dirichlet.items():
            for c in comps:
                mask[c * self.Nn:(c + 1) * self.Nn] |= on[f]
        return mask

    def lattice_coords(self, basis_nodes=None):
        """Physical coordinates of the lattice points for a nodal basis with
        1D reference nodes ``basis_nodes`` (lattice order).  Used only to
        place nodal values; modal coefficients have no coordinates."""
        P = self.P
        xs = []
        for d in range(3):
            pts = np.empty(self.N[d])
            for e in range(self.ne[d]):
                for j in range(P + 1):
                    pts[e * P + j] = (e + 0.5 * (1.0 + basis_nodes[j])) * self.h[d]
            xs.append(pts)
        return xs
