"""Pins for the oracle's element and global operators.  CPU only."""
import numpy as np
import pytest

from oracle.assembly import Discretization
from oracle.basis1d import KINDS, Basis1D
from oracle.hexmesh import BoxMesh
from oracle import material
from oracle.material import lame
from synthetic import random_vector

MU, LAM = lame(1000.0, 0.3)


def _disc(kind, P=2, elems=(1, 1, 1), lengths=(1.0, 1.0, 1.0)):
    return Discretization(BoxMesh(*elems, P, lengths), Basis1D(P, kind), MU, LAM, rho=1.3)


@pytest.mark.parametrize("kind", KINDS)
def test_internal_force_is_energy_gradient(kind):
    d = _disc(kind, P=2, lengths=(1.0, 0.7, 1.2))
    u = random_vector(d.mesh.ndof, 1, 0.02)
    R = d.internal_force(u)
    h = 1e-6
    idx = np.random.default_rng(0).choice(d.mesh.ndof, 12, replace=False)
    for i in idx:
        e = np.zeros(d.mesh.ndof)
        e[i] = h
        fd = (d.energy(u + e) - d.energy(u - e)) / (2 * h)
        assert abs(R[i] - fd) < 1e-7 * max(1.0, np.abs(R).max())


@pytest.mark.parametrize("kind", KINDS)
def test_tangent_is_force_derivative_and_symmetric(kind):
    d = _disc(kind, P=3, elems=(2, 1, 1))
    u = random_vector(d.mesh.ndof, 2, 0.01)
    x = random_vector(d.mesh.ndof, 3)
    y = random_vector(d.mesh.ndof, 4)
    h = 1e-6
    fd = (d.internal_force(u + h * x) - d.internal_force(u - h * x)) / (2 * h)
    Kx = d.tangent_apply(u, x)
    assert np.allclose(Kx, fd, rtol=1e-6, atol=1e-6 * np.abs(Kx).max())
    assert np.isclose(y @ d.tangent_apply(u, x), x @ d.tangent_apply(u, y), rtol=1e-11)
    # dense element tangent agrees with the matrix-free action
    K = d.tangent_matrix(u, b1=0.0, masked=False)
    assert np.allclose(K @ x, Kx, rtol=1e-11, atol=1e-11 * np.abs(Kx).max())


@pytest.mark.parametrize("kind", KINDS)
def test_rigid_motions_give_zero_force(kind):
    d = _disc(kind, P=2, elems=(2, 1, 1), lengths=(2.0, 1.0, 1.0))
    assert np.abs(d.internal_force(np.zeros(d.mesh.ndof))).max() == 0.0
    th = 0.5
    R = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    c = np.array([0.3, -0.2, 0.1])
    u = d.l2_project(lambda X, t: X @ (R - np.eye(3)).T + c)
    assert np.abs(d.internal_force(u)).max() < 1e-9


@pytest.mark.parametrize("kind", KINDS)
def test_mass_total_and_symmetry(kind):
    d = _disc(kind, P=3, elems=(1, 2, 1), lengths=(1.0, 2.0, 0.5))
    one = d.l2_project(lambda X, t: np.ones_like(X))
    Mx = d.mass_apply(one)
    # sum over one component of 1^T M 1 = rho |Omega|
    vol = 1.0 * 2.0 * 0.5
    assert np.isclose(one[: d.mesh.Nn] @ Mx[: d.mesh.Nn], 1.3 * vol, rtol=1e-12)
    x, y = random_vector(d.mesh.ndof, 5), random_vector(d.mesh.ndof, 6)
    assert np.isclose(y @ d.mass_apply(x), x @ d.mass_apply(y), rtol=1e-12)


@pytest.mark.parametrize("kind", ["modal", "sdme_h"])
def test_diagonal_matches_assembled(kind):
    d = _disc(kind, P=2, elems=(2, 2, 1))
    d.mesh.clamp("xmin")
    d.mask = d.mesh.constrained()
    u = random_vector(d.mesh.ndof, 7, 0.01)
    K = d.tangent_matrix(u, b1=37.0)
    assert np.allclose(d.diagonal(u, 37.0), K.diagonal(), rtol=1e-12)
    x = random_vector(d.mesh.ndof, 8)
    assert np.allclose(K @ x, d.effective_apply(u, x, 37.0), rtol=1e-11, atol=1e-10)


def test_dof_counts_static_table():
    # Table Static_error: 3[(2P+1)^3 - (2P+1)^2] free DOFs for 2x2x2 hexes
    for P, want in ((2, 300), (4, 1944), (6, 6084), (8, 13872)):
        m = BoxMesh(2, 2, 2, P).clamp("xmin")
        assert int((~m.constrained()).sum()) == want


@pytest.mark.parametrize("kind,P", [("sdme_h", 4), ("nodal", 3), ("modal", 2)])
def test_element_quadratic_form_equals_gauss_point_sum(kind, P):
    # x_e . ((K_T(u) + b1 M) x)_e of one element equals the Gauss-point sum
    # sum_q w_q (grad x : A grad x + b1 rho |x(q)|^2): the divergence and the
    # projection are the weighted adjoints of the gradient and the values.
    # The float32 tangent kernel takes p.(A p) for the PCG step length in this
    # form instead of re-reading p after the scatter.
    d = _disc(kind, P=P, elems=(2, 1, 1), lengths=(1.0, 0.8, 1.1))
    u = random_vector(d.mesh.ndof, 5, 0.01)
    x = random_vector(d.mesh.ndof, 6)
    b1 = 37.0
    U, X = d.gather(u), d.gather(x)
    ref = d.ref
    Y = ref.tangent_action(U, X, d.mu, d.lam) + b1 * ref.mass_action(X, d.rho)
    lhs = np.einsum("ecm,ecm->e", X, Y)
    A = material.tangent(ref.deformation(U), d.mu, d.lam)
    GX = ref.grad(X)
    dP = np.einsum("eqiJkL,eqkL->eqiJ", A, GX)
    VX = ref.values(X)
    rhs = (np.einsum("eqiJ,eqiJ,q->e", GX, dP, ref.w)
           + b1 * d.rho * np.einsum("eqc,eqc,q->e", VX, VX, ref.w))
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(lhs).max())
    # summed over elements it is x . (K x) of the assembled operator
    assert np.isclose(lhs.sum(), x @ (d.tangent_apply(u, x) + b1 * d.mass_apply(x)), rtol=1e-11)
