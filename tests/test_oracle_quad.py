"""Pins for the oracle's plane-strain quadrilateral discretisation (2D
tensor products, eq. ProdTensorialQuadrado).  CPU only.

The strongest pin relates it to the 3D hexahedral discretisation (pinned
separately): a 2D field extruded through one layer of hexahedra, with the
out-of-plane component zero and the in-plane components constant in z,
gives in-plane 3D internal forces and tangent actions equal to the 2D ones
times the z-integral of each z-mode.  A dropped term or a wrong index in the 2D
operators breaks that identity."""
import numpy as np
import pytest

from oracle import quad
from oracle.assembly import Discretization
from oracle.basis1d import Basis1D
from oracle.hexmesh import BoxMesh
from oracle.material import lame
from oracle.quadrature import gauss_legendre

MU, LAM = lame(1000.0, 0.3)


def _kappa(basis):
    """Coefficients of the constant function 1 in the 1D basis (lattice order)
    and the z-integrals of the modes, both from exact quadrature."""
    x, w = gauss_legendre(basis.P + 2)
    B, _ = basis.tables(x)
    M1 = B.T @ (w[:, None] * B)
    I = w @ B
    return np.linalg.solve(M1, I), I


def _extrude(u2, m2, m3, kappa):
    Nx, Ny = m2.N
    Nz = m3.N[2]
    u3 = np.zeros(m3.ndof)
    for c in range(2):
        plane = u2[c * m2.Nn:(c + 1) * m2.Nn].reshape(Ny, Nx)
        u3[c * m3.Nn:(c + 1) * m3.Nn] = (kappa[:, None, None] * plane[None]).reshape(-1)
    return u3


@pytest.mark.parametrize("kind,P", [("nodal", 2), ("sdme_h", 3), ("modal", 4)])
def test_plane_strain_equals_extruded_3d(kind, P):
    b = Basis1D(P, kind)
    m2 = quad.RectMesh(2, 1, P, lengths=(1.0, 0.7))
    m3 = BoxMesh(2, 1, 1, P, lengths=(1.0, 0.7, 0.4))
    d2 = quad.Discretization2D(m2, b, MU, LAM)
    d3 = Discretization(m3, b, MU, LAM)
    kappa, I = _kappa(b)
    rng = np.random.default_rng(P)
    u2 = 0.02 * rng.standard_normal(m2.ndof)
    x2 = rng.standard_normal(m2.ndof)
    u3, x3 = _extrude(u2, m2, m3, kappa), _extrude(x2, m2, m3, kappa)
    hz2 = 0.5 * m3.h[2]
    for R2, R3 in ((d2.internal_force(u2), d3.internal_force(u3)),
                   (d2.tangent_apply(u2, x2), d3.tangent_apply(u3, x3))):
        # in-plane components; the out-of-plane one is the reaction of the
        # clamped u_z to the plane-strain stress sigma_zz
        want = np.zeros(2 * m3.Nn)
        for c in range(2):
            plane = R2[c * m2.Nn:(c + 1) * m2.Nn].reshape(m2.N[1], m2.N[0])
            want[c * m3.Nn:(c + 1) * m3.Nn] = (hz2 * I[:, None, None] * plane[None]).reshape(-1)
        assert np.abs(R3[:2 * m3.Nn] - want).max() < 1e-11 * np.abs(want).max()


def test_quad_tangent_and_force_are_derivatives():
    b = Basis1D(3, "sdme_m")
    d = quad.Discretization2D(quad.RectMesh(2, 2, 3), b, MU, LAM)
    rng = np.random.default_rng(1)
    u = 0.02 * rng.standard_normal(d.mesh.ndof)
    v = rng.standard_normal(d.mesh.ndof)
    h = 1e-6
    fd_R = (d.energy(u + h * v) - d.energy(u - h * v)) / (2 * h)
    assert abs(fd_R - d.internal_force(u) @ v) < 1e-7 * abs(fd_R)
    fd_K = (d.internal_force(u + h * v) - d.internal_force(u - h * v)) / (2 * h)
    assert np.abs(fd_K - d.tangent_apply(u, v)).max() < 1e-6 * np.abs(fd_K).max()


def test_quad_affine_patch():
    # u = G X: uniform stress, so the internal force vanishes at interior lattice points
    b = Basis1D(2, "nodal")
    m = quad.RectMesh(3, 2, 2, lengths=(1.5, 1.0))
    d = quad.Discretization2D(m, b, MU, LAM)
    from oracle.quadrature import gauss_lobatto_legendre
    xg = gauss_lobatto_legendre(2)
    X = np.array([(e + 0.5 * (1 + xg[j])) * m.h[0] for e in range(3) for j in range(3)][::1])
    xs = np.unique(np.round(X, 14))
    ys = np.unique(np.round([(e + 0.5 * (1 + xg[j])) * m.h[1] for e in range(2) for j in range(3)], 14))
    YY, XX = np.meshgrid(ys, xs, indexing="ij")
    G = np.array([[0.01, 0.02], [-0.015, 0.005]])
    u = np.concatenate([(G[c, 0] * XX + G[c, 1] * YY).ravel() for c in range(2)])
    R = d.internal_force(u).reshape(2, m.N[1], m.N[0])
    assert np.abs(R[:, 1:-1, 1:-1]).max() < 1e-10 * np.abs(R).max()


def _static_fab_2d(ne, P, kind="sdme_h"):
    # the paper's static fabricated field u = (1.9 sin x - x, 0) (Sec. 5.1) in
    # plane strain on the unit square: body force, the exact P N on the loaded
    # edges, x = 0 clamped
    from oracle import manufactured, solvers
    fld = manufactured.static_field()
    m = quad.RectMesh(ne, ne, P).clamp("xmin")
    d = quad.Discretization2D(m, Basis1D(P, kind), MU, LAM)
    f = d.body_load(fld.body_force(MU, LAM, 1.0))
    for e in ("xmax", "ymin", "ymax"):
        f = f + d.traction_field_load(e, fld.traction(e, MU, LAM))
    u, st = solvers.static_newton(d, f, tol=1e-12, linear="direct")
    assert st["converged"] and st["newton_iters"] <= 6
    return d.l2_error(u, fld.displacement)


def test_edge_traction_field_reduces_to_uniform_and_body_load_to_area():
    m = quad.RectMesh(2, 3, 3, (1.3, 0.7))
    d = quad.Discretization2D(m, Basis1D(3, "nodal"), 1.0, 1.0)
    t = np.array([0.3, -1.1])
    for e in quad.EDGES:
        assert np.allclose(d.traction_field_load(e, lambda X, tt: np.broadcast_to(t, X.shape)),
                           d.traction_load(e, t), atol=1e-15)
    f = d.body_load(lambda X, tt: np.broadcast_to(t, X.shape))
    # nodal basis: partition of unity, so each component sums to b_c x area
    assert np.allclose([f[:m.Nn].sum(), f[m.Nn:].sum()], t * 1.3 * 0.7, rtol=1e-13)


def test_static_fabricated_field_converges_in_p_and_h():
    errs = [_static_fab_2d(2, P) for P in range(1, 6)]
    for a, b in zip(errs, errs[1:]):
        # spectral in P on a fixed 2 x 2 mesh: the x-component carries the
        # fabricated field; the y-component (exactly zero in the field) is the
        # Poisson coupling's discretisation error and is bounded by x's
        assert b[0] < a[0] / 10.0
        assert np.hypot(*b) < np.hypot(*a) / 10.0
    assert all(e[1] <= e[0] for e in errs)
    assert errs[-1][0] < 1e-7
    eh = [_static_fab_2d(ne, 2) for ne in (1, 2, 4)]
    rates = [np.log2(a[0] / b[0]) for a, b in zip(eh, eh[1:])]
    assert 2.8 < rates[-1] < 3.3                # L2 rate P + 1 at P = 2
