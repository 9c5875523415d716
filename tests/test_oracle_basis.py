"""Pins for the oracle's 1D bases (Sec. 2 of the paper).  CPU only."""
import numpy as np
import pytest

from oracle.basis1d import KINDS, Basis1D, StandardBasis, matrices_1d, simultaneous_diagonalisation
from oracle.quadrature import gauss_legendre

ORDERS = [2, 3, 4, 6, 8]


def test_modal_closed_forms():
    # linear hat vertex block of the modal basis (eq. BasePadrao1D):
    # M_vv = [[2/3, 1/3], [1/3, 2/3]], K_vv = [[1/2, -1/2], [-1/2, 1/2]]
    M, K = matrices_1d(StandardBasis(6, "modal"))
    assert np.allclose(M[:2, :2], [[2 / 3, 1 / 3], [1 / 3, 2 / 3]], atol=1e-15)
    assert np.allclose(K[:2, :2], [[0.5, -0.5], [-0.5, 0.5]], atol=1e-15)
    # the hats are K-orthogonal to every bubble, and with alpha = beta = 1 the
    # bubbles' stiffness block is diagonal (d/dx of (1-x^2) P^{1,1}_n is a
    # multiple of the Legendre polynomial L_{n+1})
    assert np.abs(K[:2, 2:]).max() < 1e-15
    off = K[2:, 2:] - np.diag(np.diag(K[2:, 2:]))
    assert np.abs(off).max() < 1e-14
    # first bubble (1-x^2)/4: int ((x/2))^2 = 1/6 ; int ((1-x^2)/4)^2 = 1/15
    assert abs(K[2, 2] - 1.0 / 6.0) < 1e-15 and abs(M[2, 2] - 1.0 / 15.0) < 1e-15


@pytest.mark.parametrize("P", ORDERS)
@pytest.mark.parametrize("k", [0.0, 0.5, 1.0])
def test_simultaneous_diagonalisation(P, k):
    M, K = matrices_1d(StandardBasis(P, "modal"))
    Y, lamS = simultaneous_diagonalisation(M, K, k)
    Mp = Y @ M[2:, 2:] @ Y.T
    Kp = Y @ K[2:, 2:] @ Y.T
    # eq. ParametroK
    assert np.allclose(Mp, np.diag(lamS ** -k), atol=1e-13 * max(1, lamS.max() ** k))
    assert np.allclose(Kp, np.diag(lamS ** (1 - k)), rtol=1e-12, atol=1e-12 * lamS.max())
    if k == 0.0:
        assert np.allclose(Mp, np.eye(P - 1), atol=1e-13)
    if k == 1.0:
        assert np.allclose(Kp, np.eye(P - 1), atol=1e-12)
    if k == 0.5:
        assert np.isclose(np.linalg.cond(Mp), np.linalg.cond(Kp), rtol=1e-10)


def test_sd_eigenvalues_are_dirichlet_laplacian():
    # L's eigenvalues are the Rayleigh-Ritz approximations of -u'' = l u on
    # [-1, 1] with u(+-1) = 0, exact eigenvalues (j pi / 2)^2, from above.
    b = Basis1D(14, "sdme_m")
    exact = (np.arange(1, 14) * np.pi / 2) ** 2
    assert np.all(b.lambda_S >= exact * (1 - 1e-12))
    assert np.allclose(b.lambda_S[:3], exact[:3], rtol=1e-9)


@pytest.mark.parametrize("P", ORDERS)
def test_minimum_energy_decoupling(P):
    lam = 100.0
    for kind, which in (("sdme_m", "M"), ("sdme_k", "K"), ("sdme_h", "H")):
        b = Basis1D(P, kind, k=0.5, lam=lam)
        M, K = b.matrices()
        G = {"M": M, "K": K, "H": K + lam * M}[which]
        scale = np.abs(G).max()
        assert np.abs(G[:2, 2:]).max() < 1e-13 * scale, kind
        # SD part: internal block of M and K stays diagonal after ME
        for A in (M, K):
            off = A[2:, 2:] - np.diag(np.diag(A[2:, 2:]))
            assert np.abs(off).max() < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("P", ORDERS)
def test_vertex_delta_and_internal_zero(kind, P):
    b = Basis1D(P, kind)
    V, _ = b.eval(np.array([-1.0, 1.0]))
    assert np.allclose(V[0], [1, 0], atol=1e-13)
    assert np.allclose(V[1], [0, 1], atol=1e-13)
    assert np.abs(V[2:]).max() < 1e-13


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("P", ORDERS)
def test_span_and_linear_reproduction(kind, P):
    b = Basis1D(P, kind)
    x, w = gauss_legendre(P + 3)
    V, _ = b.eval(x)
    # change of basis to monomials has full rank: span is P_P
    mono = np.vander(x, P + 1, increasing=True).T
    C = np.linalg.lstsq(V.T, mono.T, rcond=None)[0]
    assert np.linalg.matrix_rank(C) == P + 1
    assert np.allclose(V.T @ C, mono.T, atol=1e-11)
    # constant and linear functions are reproduced by the full expansion
    for f in (np.ones_like(x), x):
        c = np.linalg.lstsq(V.T, f, rcond=None)[0]
        assert np.allclose(V.T @ c, f, atol=1e-12)


@pytest.mark.parametrize("P", ORDERS)
def test_partition_of_unity(P):
    x = np.linspace(-1, 1, 11)
    # the Lagrange set sums to one as a whole (its vertex pair alone does not)
    V, _ = Basis1D(P, "nodal").eval(x)
    assert np.allclose(V.sum(axis=0), 1.0, atol=1e-12)
    # vertex pairs of the modal and SDME-K bases are the linear hats
    for kind in ("modal", "sdme_k"):
        V, _ = Basis1D(P, kind).eval(x)
        assert np.allclose(V[0] + V[1], 1.0, atol=1e-12), kind
    for kind in ("sdme_m", "sdme_h"):
        V, _ = Basis1D(P, kind).eval(x)
        assert np.abs(V[0] + V[1] - 1.0).max() > 1e-3, kind


@pytest.mark.parametrize("kind", ["sdme_m", "sdme_k", "sdme_h"])
@pytest.mark.parametrize("P", ORDERS)
def test_sdme_start_independent(kind, P):
    # SD modes are the pencil's eigenfunctions and ME vertex modes are
    # projections; neither depends on the standard basis they start from.
    x = np.linspace(-1, 1, 9)
    a = Basis1D(P, kind, start="modal").eval(x)
    b = Basis1D(P, kind, start="nodal").eval(x)
    assert np.allclose(a[0], b[0], atol=1e-11) and np.allclose(a[1], b[1], atol=1e-9)


@pytest.mark.parametrize("kind", ["sdme_m", "sdme_h"])
def test_me_with_transformed_internal_modes(kind):
    # eq. ExtensaoMEmassa with the SD-transformed internal functions gives
    # the same vertex functions as with the original ones.
    P, lam = 6, 100.0
    b = Basis1D(P, kind, lam=lam)
    M, K = b.M_std, b.K_std
    Y = b.T[2:, 2:]
    Tn = np.eye(P + 1)
    Tn[2:, 2:] = Y
    Mt, Kt = Tn @ M @ Tn.T, Tn @ K @ Tn.T
    G = Mt if kind == "sdme_m" else Kt + lam * Mt
    alpha_t = np.linalg.solve(G[2:, 2:].T, G[:2, 2:].T).T
    x = np.linspace(-1, 1, 9)
    V, _ = b.std.eval(x)
    phi_t = V[:2] - alpha_t @ (Y @ V[2:])
    phi, _ = b.eval(x)
    assert np.allclose(phi_t, phi[:2], atol=1e-12)


@pytest.mark.parametrize("P", ORDERS)
def test_sign_convention(P):
    b = Basis1D(P, "sdme_h")
    _, D = b.eval(np.array([-1.0]))
    assert np.all(D[2:, 0] > 0)


def test_lattice_order():
    b = Basis1D(4, "modal")
    B, D = b.tables(np.array([-1.0, 1.0]))
    assert np.allclose(B[0], [1, 0, 0, 0, 0]) and np.allclose(B[1], [0, 0, 0, 0, 1])
