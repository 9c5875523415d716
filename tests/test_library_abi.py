"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/sdme.h declares, and its host-only basis builder agrees with the
oracle.  No GPU call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sdme.h")
LIB = os.path.join(ROOT, "paper_2104_13466_gb300", "libsdme.so")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:sdme_status|const char\*|int)\s+(sdme_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__._build_module().build(verbose=False)
    return ctypes.CDLL(LIB)


def test_header_declares_entry_points():
    names = _declared()
    for required in ("sdme_build_basis1d", "sdme_create", "sdme_destroy", "sdme_internal_force",
                     "sdme_tangent_apply", "sdme_pcg_solve", "sdme_implicit_newmark_step"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib):
    import paper_2104_13466_gb300 as s
    assert sorted(s.EXPORTS) == _declared()


@pytest.mark.parametrize("kind", ["nodal", "modal", "sdme_m", "sdme_k", "sdme_h"])
@pytest.mark.parametrize("P", [1, 2, 3, 5, 8])
def test_host_basis_builder_matches_oracle(kind, P):
    # sdme_build_basis1d is a host-only routine (no device work)
    import paper_2104_13466_gb300 as s
    from oracle.basis1d import Basis1D
    from oracle.quadrature import gauss_legendre
    xq, wq, B, D, M1, K1 = s.build_basis1d(P, kind)
    b = Basis1D(P, kind)
    x2, w2 = gauss_legendre(P + 2)
    B2, D2 = b.tables(x2)
    o = b.lattice_order
    M2, K2 = [m[np.ix_(o, o)] for m in b.matrices()]
    assert np.allclose(xq, x2, atol=1e-15) and np.allclose(wq, w2, atol=1e-15)
    assert np.abs(B - B2).max() < 1e-12 * max(1, np.abs(B2).max())
    assert np.abs(D - D2).max() < 1e-11 * max(1, np.abs(D2).max())
    assert np.abs(M1 - M2).max() < 1e-12 * np.abs(M2).max()
    assert np.abs(K1 - K2).max() < 1e-11 * np.abs(K2).max()


def test_basis_builder_rejects_bad_input(lib):
    import paper_2104_13466_gb300 as s
    with pytest.raises(s.SdmeError):
        s.build_basis1d(9, "sdme_h")
    with pytest.raises(s.SdmeError):
        s.build_basis1d(4, "sdme_h", k=2.0)
