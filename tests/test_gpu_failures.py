"""Failure detection through the C ABI, with every failure made on the host
(no test here faults, traps or hangs a GPU):

* a NaN written from the host into an input vector -> SDME_NAN (the PCG
  breakdown test and the Newton residual norm), the Newmark state left at t_n;
* maxit = 1 -> SDME_PCG_MAXIT after exactly one iteration, in both precisions;
* max_newton = 1 on a step that needs more -> SDME_NEWTON_DIVERGED, with u, v
  and a bit-for-bit unchanged;
* corrupt mesh, material and basis descriptors -> SDME_EINVAL from
  sdme_create, with no context returned.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.material import lame  # noqa: E402
from synthetic import random_vector  # noqa: E402


def _sdme():
    import paper_2104_13466_gb300 as s
    return s


def _ctx(prec=0, P=3):
    s = _sdme()
    mu, lam = lame(1000.0, 0.3)
    return s.Context((3, 2, 2), (1.5, 1.0, 1.0), {"xmin": (0, 1, 2)}, mu, lam, 1.0, P, "sdme_h", precision=prec)


def _load(ctx, mag=-50.0):
    f = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.traction_load("xmax", (0.0, 0.0, mag), f)
    return f


@pytest.mark.parametrize("prec", [0, 1])
def test_nan_in_right_hand_side_is_reported(prec):
    s = _sdme()
    ctx = _ctx(prec)
    b = torch.from_numpy(random_vector(ctx.ndof, 3)).cuda()
    b[ctx.ndof // 2 + 7] = float("nan")          # a free DOF (x = 0 is the clamped face)
    x = torch.zeros_like(b)
    u = torch.zeros_like(b)
    with pytest.raises(s.SdmeError) as e:
        ctx.pcg_solve(u, 10.0, b, x, rtol=1e-10, maxit=100)
    assert e.value.status == s.NAN
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_nan_in_load_leaves_state_at_t_n(prec):
    s = _sdme()
    ctx = _ctx(prec)
    f = _load(ctx)
    u, v, a = (torch.from_numpy(random_vector(ctx.ndof, k, 1e-4)).cuda() for k in (4, 5, 6))
    for t in (u, v, a):
        t[:: ctx.N[0]] = 0.0                      # clamped lattice points (ix = 0) hold 0
    u0, v0, a0 = u.clone(), v.clone(), a.clone()
    f[ctx.ndof - 5] = float("nan")
    st = ctx.implicit_newmark_step(u, v, a, 0.01, f, allow=(s.NAN,))
    assert st["status"] == s.NAN and not st["converged"]
    assert torch.equal(u, u0) and torch.equal(v, v0) and torch.equal(a, a0)
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_pcg_maxit_one(prec):
    s = _sdme()
    ctx = _ctx(prec)
    b = torch.from_numpy(random_vector(ctx.ndof, 8)).cuda()
    x = torch.zeros_like(b)
    u = torch.zeros_like(b)
    with pytest.raises(s.SdmeError) as e:
        ctx.pcg_solve(u, 10.0, b, x, rtol=1e-12, maxit=1)
    assert e.value.status == s.PCG_MAXIT
    its, rel = ctx.pcg_solve(u, 10.0, b, x, rtol=1e-12, maxit=1, allow_maxit=True)
    assert its == 1 and np.isfinite(rel) and rel > 0.0
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_max_newton_one_diverges_and_keeps_state(prec):
    s = _sdme()
    ctx = _ctx(prec)
    f = _load(ctx, mag=-200.0)
    u, v, a = (torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda") for _ in range(3))
    st = ctx.implicit_newmark_step(u, v, a, 0.01, f, max_newton=1, newton_tol=1e-10, allow=(s.NEWTON_DIVERGED,))
    assert st["status"] == s.NEWTON_DIVERGED and not st["converged"] and st["newton_iters"] == 1
    assert st["residual_rel"] > 1e-10
    assert not torch.any(u) and not torch.any(v) and not torch.any(a)
    with pytest.raises(s.SdmeError) as e:
        ctx.implicit_newmark_step(u, v, a, 0.01, f, max_newton=1, newton_tol=1e-10)
    assert e.value.status == s.NEWTON_DIVERGED
    # the same step with enough iterations converges from the kept state
    st = ctx.implicit_newmark_step(u, v, a, 0.01, f, newton_tol=1e-10)
    assert st["converged"] and st["newton_iters"] > 1
    ctx.close()


def _create(mesh, mat=None, basis=None, prec=0):
    s = _sdme()
    mat = mat or s.Material(384.6, 576.9, 1.0)
    basis = basis or s.basis_desc(3, "sdme_h")
    h = ctypes.c_void_p()
    st = s.lib.sdme_create(ctypes.byref(h), ctypes.byref(mesh) if mesh is not None else None,
                           ctypes.byref(mat), ctypes.byref(basis), prec, None)
    if h.value:
        s.lib.sdme_destroy(h)
    return st, h.value


def _mesh(elems=(2, 2, 2), lengths=(1.0, 1.0, 1.0), clamp=None):
    s = _sdme()
    m = s.MeshDesc()
    for d in range(3):
        m.nelem[d] = elems[d]
        m.length[d] = lengths[d]
    for f, bits in (clamp or {}).items():
        m.clamp[f] = bits
    return m


@pytest.mark.parametrize("case", ["negative_count", "zero_length", "nan_length", "inf_length", "overflow",
                                  "2d_with_z_clamp", "null_mesh", "bad_material", "bad_precision",
                                  "bad_basis_order", "bad_basis_kind", "bad_sd_parameter"])
def test_corrupt_descriptors_rejected(case):
    s = _sdme()
    mesh, mat, basis, prec = _mesh(), None, None, 0
    if case == "negative_count":
        mesh = _mesh(elems=(2, -3, 2))
    elif case == "zero_length":
        mesh = _mesh(lengths=(1.0, 0.0, 1.0))
    elif case == "nan_length":
        mesh = _mesh(lengths=(float("nan"), 1.0, 1.0))
    elif case == "inf_length":
        mesh = _mesh(lengths=(1.0, float("inf"), 1.0))
    elif case == "overflow":
        mesh = _mesh(elems=(1 << 20, 1 << 20, 1 << 20))
    elif case == "2d_with_z_clamp":
        mesh = _mesh(elems=(2, 2, 0), clamp={4: 7})
    elif case == "null_mesh":
        mesh = None
    elif case == "bad_material":
        mat = s.Material(-1.0, 576.9, 1.0)
    elif case == "bad_precision":
        prec = 7
    elif case == "bad_basis_order":
        basis = s.basis_desc(3, "sdme_h")
        basis.P = 12
    elif case == "bad_basis_kind":
        basis = s.basis_desc(3, "sdme_h")
        basis.kind = 42
    elif case == "bad_sd_parameter":
        basis = s.basis_desc(3, "sdme_h", k=1.5)
    st, h = _create(mesh, mat, basis, prec)
    assert st == s.EINVAL and not h
