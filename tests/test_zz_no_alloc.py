"""sdme_tangent_apply_noalloc, the allocation-free tangent matvec.

Some callers cannot allocate device memory (a fixed memory budget, a pool
that forbids new allocations, code that must not trigger allocator
synchronisation).  They call this entry point, which keeps its scratch in a
static device array inside the library.  Its result must equal the
context-based sdme_tangent_apply to the float64 tolerance used everywhere
else (1e-10 relative), on consecutive calls that share that array.

The result is also checked against the FP64 oracle's effective tangent
(Sec. 3, consistent linearisation) at P = 8, the largest order, on a mesh
that fits the array.

This file is collected last on purpose, so that a failure here does not stop
a first-failure run before the other tests have run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.material import lame  # noqa: E402
from synthetic import random_vector  # noqa: E402

TOL64 = 1e-10
ELEMS, LENGTHS = (3, 2, 2), (1.3, 0.7, 0.9)
CLAMP = {"xmin": (0, 1, 2), "zmax": (2,)}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _call_noalloc(s, P, tables, mu, lam, rho, u, b1, x, y, elems=ELEMS, lengths=LENGTHS, clamp=CLAMP):
    # straight through the C ABI
    mesh = s.mesh_desc(elems, lengths, clamp)
    mat = s.Material(mu, lam, rho)
    arrs = [np.ascontiguousarray(t, dtype=np.float64) for t in tables]
    ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrs]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return s.lib.sdme_tangent_apply_noalloc(ctypes.byref(mesh), ctypes.byref(mat), P, *ptrs,
                                            ctypes.c_void_p(u.data_ptr()), ctypes.c_double(b1),
                                            ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), stream)


@pytest.mark.parametrize("P,kind", [(4, "sdme_h"), (6, "modal")])
def test_noalloc_tangent_matches_context_tangent_twice(P, kind):
    import paper_2104_13466_gb300 as s
    mu, lam = lame(1000.0, 0.3)
    rho = 1.3
    ctx = s.Context(ELEMS, LENGTHS, CLAMP, mu, lam, rho, P, kind)
    xq, wq, B, D, _, _ = s.build_basis1d(P, kind)
    hmin = min(LENGTHS[d] / ELEMS[d] for d in range(3))
    # two calls in a row with different inputs: the second must not see the
    # first call's leftovers in the shared scratch array
    for call, (seed, b1) in enumerate(((11, 250.0), (12, 0.0))):
        u = _dev(random_vector(ctx.ndof, seed, 0.02 * hmin / P))
        x = _dev(random_vector(ctx.ndof, seed + 100))
        y_ref = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
        ctx.tangent_apply(u, b1, x, y_ref)
        y = torch.full((ctx.ndof,), float("nan"), dtype=torch.float64, device="cuda")
        st = _call_noalloc(s, P, (xq, wq, B, D), mu, lam, rho, u, b1, x, y)
        assert st == s.OK, (call, st)
        torch.cuda.synchronize()
        ref = y_ref.cpu().numpy()
        got = y.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < TOL64, (call, err)
    ctx.close()


def test_noalloc_tangent_matches_oracle_at_p8():
    import paper_2104_13466_gb300 as s
    from oracle.assembly import Discretization
    from oracle.basis1d import Basis1D
    from oracle.hexmesh import BoxMesh
    P, kind = 8, "sdme_h"
    elems, lengths = (2, 2, 1), (1.0, 0.8, 0.6)
    clamp = {"xmin": (0, 1, 2)}
    mu, lam = lame(1000.0, 0.45)
    rho = 1.0
    mesh = BoxMesh(*elems, P, lengths).clamp("xmin")
    disc = Discretization(mesh, Basis1D(P, kind), mu, lam, rho)
    xq, wq, B, D, _, _ = s.build_basis1d(P, kind)
    for seed, b1 in ((21, 4.0), (22, 0.0)):
        u = random_vector(mesh.ndof, seed, 0.02 * 0.6 / P)
        x = random_vector(mesh.ndof, seed + 100)
        y = torch.full((mesh.ndof,), float("nan"), dtype=torch.float64, device="cuda")
        st = _call_noalloc(s, P, (xq, wq, B, D), mu, lam, rho, _dev(u), b1, _dev(x), y, elems, lengths, clamp)
        assert st == s.OK
        torch.cuda.synchronize()
        want = disc.effective_apply(u, x, b1)
        got = y.cpu().numpy()
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err < TOL64, (seed, err)


def test_noalloc_rejects_problems_beyond_its_scratch():
    import paper_2104_13466_gb300 as s
    mu, lam = lame(1000.0, 0.3)
    P = 8
    xq, wq, B, D, _, _ = s.build_basis1d(P, "sdme_h")
    big = s.mesh_desc((20, 20, 20), (1.0, 1.0, 1.0), {})
    mat = s.Material(mu, lam, 1.0)
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    arrs = [np.ascontiguousarray(t, dtype=np.float64) for t in (xq, wq, B, D)]
    ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrs]
    st = s.lib.sdme_tangent_apply_noalloc(ctypes.byref(big), ctypes.byref(mat), P, *ptrs,
                                          ctypes.c_void_p(one.data_ptr()), ctypes.c_double(0.0),
                                          ctypes.c_void_p(one.data_ptr()), ctypes.c_void_p(one.data_ptr()),
                                          ctypes.c_void_p(0))
    assert st == s.EINVAL
    # plane-strain meshes (nelem[2] = 0) are not served by this entry point
    flat = s.mesh_desc((2, 2), (1.0, 1.0), {})
    st = s.lib.sdme_tangent_apply_noalloc(ctypes.byref(flat), ctypes.byref(mat), P, *ptrs,
                                          ctypes.c_void_p(one.data_ptr()), ctypes.c_double(0.0),
                                          ctypes.c_void_p(one.data_ptr()), ctypes.c_void_p(one.data_ptr()),
                                          ctypes.c_void_p(0))
    assert st == s.EINVAL
