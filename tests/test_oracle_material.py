"""Pins for the oracle's neo-Hookean law (Sec. 3, eqs. hyperelastic strain
energy and second Piolla_Kirchhoff relation).  CPU only."""
import numpy as np
import pytest

from oracle import material

MU, LAM = material.lame(1000.0, 0.3)


def _random_F(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    F = np.eye(3) + scale * rng.standard_normal((3, 3))
    assert np.linalg.det(F) > 0
    return F


def test_lame():
    mu, lam = material.lame(1000.0, 0.3)
    assert np.isclose(mu, 384.6153846153846) and np.isclose(lam, 576.9230769230769)


@pytest.mark.parametrize("seed", range(4))
def test_pk1_is_energy_gradient(seed):
    F = _random_F(seed)
    P = material.pk1(F, MU, LAM)
    h = 1e-6
    G = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            E = np.zeros((3, 3))
            E[i, j] = h
            G[i, j] = (material.energy(F + E, MU, LAM) - material.energy(F - E, MU, LAM)) / (2 * h)
    assert np.allclose(P, G, rtol=1e-7, atol=1e-6)


@pytest.mark.parametrize("seed", range(4))
def test_tangent_is_stress_derivative(seed):
    F = _random_F(seed + 10)
    A = material.tangent(F, MU, LAM)
    h = 1e-6
    for k in range(3):
        for l in range(3):
            E = np.zeros((3, 3))
            E[k, l] = h
            fd = (material.pk1(F + E, MU, LAM) - material.pk1(F - E, MU, LAM)) / (2 * h)
            assert np.allclose(A[:, :, k, l], fd, rtol=1e-6, atol=1e-5)
    # major symmetry of a hyperelastic tangent
    assert np.allclose(A, A.transpose(2, 3, 0, 1), atol=1e-9)


def test_reference_state_and_small_strain_limit():
    I = np.eye(3)
    assert np.allclose(material.pk1(I, MU, LAM), 0.0, atol=1e-12)
    assert np.allclose(material.tangent(I, MU, LAM), material.linear_elastic_tangent(MU, LAM), atol=1e-10)


def test_frame_invariance_and_balance():
    F = _random_F(3)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    assert np.isclose(material.energy(R @ F, MU, LAM), material.energy(F, MU, LAM))
    assert np.allclose(material.pk1(R @ F, MU, LAM), R @ material.pk1(F, MU, LAM), atol=1e-10)
    assert np.allclose(material.pk1(R, MU, LAM), 0.0, atol=1e-10)
    # Kirchhoff stress P F^T is symmetric
    tau = material.pk1(F, MU, LAM) @ F.T
    assert np.allclose(tau, tau.T, atol=1e-10)


def test_uniaxial_closed_form():
    # F = diag(s, 1, 1): P_xx = mu (s - 1/s) + lambda ln s / s, P_yy = lambda ln s
    s = 1.3
    P = material.pk1(np.diag([s, 1.0, 1.0]), MU, LAM)
    assert np.isclose(P[0, 0], MU * (s - 1 / s) + LAM * np.log(s) / s)
    assert np.isclose(P[1, 1], LAM * np.log(s)) and np.isclose(P[2, 2], LAM * np.log(s))
