"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: float64 kernels 1e-10 relative (max-norm of the difference over
max-norm of the oracle result).  Float32 (SDME_MIXED_FP32) tangent: 2e-5
relative, from float32 unit roundoff 6e-8 times the depth of the contraction
chain (3 interpolation + 1 derivative stages forward and back, sums of
length <= 10, collocation-derivative entries up to ~Q^2) with a margin; the
measured error is reported by the test on failure.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import solvers  # noqa: E402
from oracle.assembly import Discretization, elements_touching  # noqa: E402
from oracle.basis1d import Basis1D  # noqa: E402
from oracle.hexmesh import BoxMesh  # noqa: E402
from oracle.material import lame  # noqa: E402
from synthetic import random_vector, workload, load_magnitude  # noqa: E402

TOL64 = 1e-10
TOL32 = 2e-5
KINDS = ["nodal", "modal", "sdme_m", "sdme_k", "sdme_h"]


def _sdme():
    import paper_2104_13466_gb300 as s
    return s


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _pair(elems, lengths, clamp, P, kind, prec=0, E=1000.0, nu=0.3, rho=1.3):
    s = _sdme()
    mu, lam = lame(E, nu)
    ctx = s.Context(elems, lengths, clamp, mu, lam, rho, P, kind, precision=prec)
    mesh = BoxMesh(*elems, P, lengths)
    for f, comps in clamp.items():
        mesh.clamp(f, comps)
    disc = Discretization(mesh, Basis1D(P, kind), mu, lam, rho)
    assert ctx.ndof == mesh.ndof and tuple(ctx.N) == mesh.N
    return ctx, disc


RAGGED = dict(elems=(3, 2, 2), lengths=(1.3, 0.7, 0.9), clamp={"xmin": (0, 1, 2), "zmax": (2,)})


def _u(disc, seed, amp=0.02):
    # small smooth-free random displacement: amplitude scaled by element size
    return random_vector(disc.mesh.ndof, seed, amp * min(disc.mesh.h) / max(1, disc.mesh.P))


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 7, 8])
def test_internal_force_all_orders(P):
    ctx, disc = _pair(P=P, kind="sdme_h", **RAGGED)
    u = _u(disc, 100 + P)
    R = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.internal_force(_dev(u), R)
    want = disc.internal_force(u)
    assert _relerr(_host(R), want) < TOL64


@pytest.mark.parametrize("kind", KINDS)
def test_internal_force_all_bases(kind):
    ctx, disc = _pair(P=4, kind=kind, **RAGGED)
    u = _u(disc, 7)
    R = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.internal_force(_dev(u), R)
    assert _relerr(_host(R), disc.internal_force(u)) < TOL64


@pytest.mark.parametrize("P", [1, 3, 6, 8])
def test_mass_apply(P):
    ctx, disc = _pair(P=P, kind="sdme_m", **RAGGED)
    x = random_vector(disc.mesh.ndof, 11)
    y = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.mass_apply(_dev(x), y)
    assert _relerr(_host(y), disc.mass_apply(x)) < TOL64


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("b1", [0.0, 250.0])
def test_tangent_apply_fp64(P, b1):
    ctx, disc = _pair(P=P, kind="sdme_h", **RAGGED)
    u = _u(disc, 200 + P)
    x = random_vector(disc.mesh.ndof, 300 + P)
    y = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.tangent_apply(_dev(u), b1, _dev(x), y)
    assert _relerr(_host(y), disc.effective_apply(u, x, b1)) < TOL64


@pytest.mark.parametrize("kind", KINDS)
def test_tangent_apply_bases(kind):
    ctx, disc = _pair(P=5, kind=kind, **RAGGED)
    u = _u(disc, 21)
    x = random_vector(disc.mesh.ndof, 22)
    y = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.tangent_apply(_dev(u), 40.0, _dev(x), y)
    assert _relerr(_host(y), disc.effective_apply(u, x, 40.0)) < TOL64


@pytest.mark.parametrize("P", [2, 4, 6, 8])
def test_tangent_apply_mixed(P):
    s = _sdme()
    ctx, disc = _pair(P=P, kind="sdme_h", prec=s.MIXED_FP32, **RAGGED)
    u = _u(disc, 400 + P)
    x = random_vector(disc.mesh.ndof, 500 + P)
    y = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.tangent_apply(_dev(u), 250.0, _dev(x), y)
    err = _relerr(_host(y), disc.effective_apply(u, x, 250.0))
    assert err < TOL32, err


@pytest.mark.parametrize("P", [1, 2, 4, 8])
@pytest.mark.parametrize("kind", ["modal", "sdme_h"])
def test_diagonal(P, kind):
    ctx, disc = _pair(P=P, kind=kind, **RAGGED)
    u = _u(disc, 600 + P)
    d = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.diagonal(_dev(u), 75.0, d)
    assert _relerr(_host(d), disc.diagonal(u, 75.0)) < TOL64


@pytest.mark.parametrize("kind", ["nodal", "modal", "sdme_h"])
def test_pcg_matches_dense_direct(kind):
    ctx, disc = _pair(elems=(2, 2, 1), lengths=(1.0, 1.0, 0.5), clamp={"zmin": (0, 1, 2)}, P=3, kind=kind)
    u = _u(disc, 31)
    u[disc.mask] = 0.0
    b = random_vector(disc.mesh.ndof, 32)
    b1 = 400.0
    x = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    its, rel = ctx.pcg_solve(_dev(u), b1, _dev(b), x, rtol=1e-13, maxit=5000)
    bm = np.where(disc.mask, 0.0, b)
    x_dir = solvers.dense_solve(disc.tangent_matrix(u, b1), bm)
    assert rel <= 1e-13
    assert _relerr(_host(x), x_dir) < 1e-10
    # same algorithm and stopping rule as the oracle's CGD: the same count up
    # to the last few iterations, where a tolerance this close to round-off
    # is met at an iteration that depends on the (atomic) summation order
    _, its_or, _ = solvers.jacobi_pcg(lambda v: disc.effective_apply(u, v, b1), bm, disc.diagonal(u, b1), 1e-13)
    assert abs(its - its_or) <= max(2, its_or // 50)


def test_pcg_mixed_reaches_float32_tolerance():
    s = _sdme()
    ctx, disc = _pair(elems=(2, 2, 2), lengths=(1.0, 1.0, 1.0), clamp={"zmin": (0, 1, 2)}, P=4, kind="sdme_h",
                      prec=s.MIXED_FP32)
    u = np.zeros(disc.mesh.ndof)
    b = random_vector(disc.mesh.ndof, 41)
    x = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    its, rel = ctx.pcg_solve(_dev(u), 100.0, _dev(b), x, rtol=1e-5, maxit=5000)
    bm = np.where(disc.mask, 0.0, b)
    xh = _host(x)
    r = bm - disc.effective_apply(u, xh, 100.0)
    assert np.linalg.norm(r) < 1e-4 * np.linalg.norm(bm)


@pytest.mark.parametrize("grid", [-1, 7])
@pytest.mark.parametrize("prec", [0, 1])
def test_pcg_with_a_fixed_tangent_grid(prec, grid):
    # the tangent launch with fewer CTAs than elements (each CTA serving every
    # grid-th element, one step-length partial per CTA) solves the same
    # system as one CTA per element: against the dense direct solve, with the
    # same iteration count up to the last few (summation order; the float32
    # recurrence with its float64 restarts drifts by a few per cent)
    s = _sdme()
    ctx, disc = _pair(elems=(3, 2, 2), lengths=(1.3, 0.7, 0.9), clamp={"xmin": (0, 1, 2), "zmax": (2,)}, P=4,
                      kind="sdme_h", prec=s.MIXED_FP32 if prec else 0)
    u = _u(disc, 61)
    u[disc.mask] = 0.0
    b = random_vector(disc.mesh.ndof, 62)
    b1, rtol = 300.0, (1e-6 if prec else 1e-12)
    x0 = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    its0, _ = ctx.pcg_solve(_dev(u), b1, _dev(b), x0, rtol=rtol, maxit=5000)
    used = ctx.set_tangent_grid(grid)
    assert 0 < used < disc.mesh.nelem or grid == -1
    x = torch.zeros_like(x0)
    its, rel = ctx.pcg_solve(_dev(u), b1, _dev(b), x, rtol=rtol, maxit=5000)
    assert rel <= rtol and abs(its - its0) <= (max(2, its0 // 20) if prec else 2)
    bm = np.where(disc.mask, 0.0, b)
    x_dir = solvers.dense_solve(disc.tangent_matrix(u, b1), bm)
    assert _relerr(_host(x), x_dir) < (1e-4 if prec else 1e-9)
    assert ctx.set_tangent_grid(0) == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_pcg_above_the_deferred_size(prec):
    # 9,216 elements: above the size up to which the PCG update sums the
    # operator's per-element p.(A p) partials, so here the operator's last CTA
    # forms the step length (with the table-driven gather of even orders);
    # the true residual is checked on sampled DOFs, element by element
    s = _sdme()
    ctx, disc = _pair(elems=(24, 24, 16), lengths=(1.0, 1.0, 0.7), clamp={"zmin": (0, 1, 2)}, P=2,
                      kind="sdme_h", prec=s.MIXED_FP32 if prec else 0)
    assert disc.mesh.nelem > 8192
    n = disc.mesh.ndof
    b = random_vector(n, 81)
    b1 = 100.0
    rtol = 1e-5 if prec else 1e-10
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    its, rel = ctx.pcg_solve(_dev(np.zeros(n)), b1, _dev(b), x, rtol=rtol, maxit=20000)
    assert rel <= rtol and its > 10
    xh = _host(x)
    bm = np.where(disc.mask, 0.0, b)
    dofs = np.sort(np.random.default_rng(82).choice(np.flatnonzero(~disc.mask), 64, replace=False))
    els = elements_touching(disc.mesh, dofs)
    xm = np.where(disc.mask, 0.0, xh)
    Ue, Xe = disc.gather(np.zeros(n), els), disc.gather(xm, els)
    Ye = disc.ref.tangent_action(Ue, Xe, disc.mu, disc.lam) + b1 * disc.ref.mass_action(Xe, disc.rho)
    r = bm[dofs] - disc.scatter(Ye, els)[dofs]
    assert np.abs(r).max() <= (1e-4 if prec else 1e-8) * np.linalg.norm(bm)


def _newmark_pair(prec, kind="sdme_h", steps=3):
    s = _sdme()
    w = workload("cube_p4")
    P = 3
    ctx, disc = _pair(elems=(2, 2, 2), lengths=(1.0, 1.0, 1.0), clamp={"zmin": (0, 1, 2)}, P=P, kind=kind,
                      prec=prec, E=w["E"], nu=w["nu"], rho=w["rho"])
    smag = load_magnitude(w["load_key"])
    unit = disc.traction_load("zmax", lambda X, t: np.broadcast_to([0.0, 0.0, -1.0], X.shape))
    fdev = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.traction_load("zmax", (0.0, 0.0, -1.0), fdev)
    assert _relerr(_host(fdev), unit) < 1e-12
    dt = w["dt"]
    u = np.zeros(disc.mesh.ndof)
    v = np.zeros_like(u)
    a = np.zeros_like(u)
    ud, vd, ad = _dev(u), _dev(v), _dev(a)
    for n in range(1, steps + 1):
        Pn = unit * smag * n / w["steps"]
        u, v, a, st = solvers.newmark_step(disc, u, v, a, Pn, dt, tol=1e-12, pcg_rtol=1e-13)
        assert st["converged"]
        stats = ctx.implicit_newmark_step(ud, vd, ad, dt, fdev * (smag * n / w["steps"]), newton_tol=1e-12,
                                          pcg_rtol=1e-13, mixed_rtol=1e-5)
        assert stats["converged"]
    return (u, v, a), (_host(ud), _host(vd), _host(ad)), stats


def test_newmark_steps_fp64():
    (u, v, a), (ug, vg, ag), stats = _newmark_pair(0)
    assert _relerr(ug, u) < 1e-9 and _relerr(vg, v) < 1e-8 and _relerr(ag, a) < 1e-7
    assert stats["newton_iters"] >= 1


def test_newmark_steps_mixed():
    s = _sdme()
    (u, v, a), (ug, vg, ag), stats = _newmark_pair(s.MIXED_FP32)
    # the Newton residual is float64, so the converged state matches the
    # float64 oracle to the Newton tolerance, not to float32 round-off
    assert _relerr(ug, u) < 1e-8 and _relerr(vg, v) < 1e-6


def test_zero_load_converges_immediately():
    ctx, disc = _pair(elems=(1, 1, 1), lengths=(1, 1, 1), clamp={"xmin": (0, 1, 2)}, P=2, kind="sdme_h")
    z = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    u, v, a = z.clone(), z.clone(), z.clone()
    st = ctx.implicit_newmark_step(u, v, a, 0.01, z)
    assert st["converged"] and st["newton_iters"] == 0 and st["pcg_iters_total"] == 0


def test_fully_constrained_is_identity():
    # P = 1, one element, all faces clamped: every DOF is constrained
    clamp = {f: (0, 1, 2) for f in ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")}
    ctx, disc = _pair(elems=(1, 1, 1), lengths=(1, 1, 1), clamp=clamp, P=1, kind="modal")
    x = random_vector(ctx.ndof, 5)
    y = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.tangent_apply(_dev(np.zeros(ctx.ndof)), 10.0, _dev(x), y)
    assert np.array_equal(_host(y), x)


def test_nonpositive_jacobian_is_reported():
    s = _sdme()
    ctx, disc = _pair(elems=(1, 1, 1), lengths=(1, 1, 1), clamp={}, P=2, kind="modal")
    # u = -2 X inverts the element (F = -I)
    u = disc.l2_project(lambda X, t: -2.0 * X)
    R = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(s.SdmeError) as ei:
        ctx.internal_force(_dev(u), R)
    assert ei.value.status == s.NONPOSITIVE_J
    # the context stays usable afterwards
    ctx.internal_force(_dev(np.zeros(ctx.ndof)), R)
    assert float(torch.abs(R).max()) == 0.0


def test_invalid_arguments_rejected():
    s = _sdme()
    with pytest.raises(s.SdmeError):
        s.Context((0, 1, 1), (1, 1, 1), {}, 1.0, 1.0, 1.0, 2, "modal")
    with pytest.raises(s.SdmeError):
        s.Context((1, 1, 1), (1, 1, 1), {}, 1.0, 1.0, 1.0, 9, "modal")
    with pytest.raises(s.SdmeError):
        s.Context((1, 1, 1), (1, -1, 1), {}, 1.0, 1.0, 1.0, 2, "modal")


def _full_beam(prec):
    s = _sdme()
    w = workload("beam_p8")
    mu, lam = lame(w["E"], w["nu"])
    ctx = s.Context(w["elems"], w["lengths"], w["clamp"], mu, lam, w["rho"], w["P"], "sdme_h", precision=prec)
    mesh = BoxMesh(*w["elems"], w["P"], w["lengths"])
    for f, comps in w["clamp"].items():
        mesh.clamp(f, comps)
    disc = Discretization(mesh, Basis1D(w["P"], "sdme_h"), mu, lam, w["rho"])
    return ctx, disc


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_beam_sampled_tangent(prec):
    # the 64x8x8, P = 8 cantilever (6.5 M DOFs) in the launch configuration
    # the benchmark uses; the oracle evaluates 24 sampled outputs element by
    # element
    ctx, disc = _full_beam(prec)
    n = disc.mesh.ndof
    u = random_vector(n, 71, 1e-4)
    x = random_vector(n, 72)
    b1 = 4.0
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.tangent_apply(_dev(u), b1, _dev(x), y)
    yg = _host(y)
    rng = np.random.default_rng(73)
    dofs = np.sort(rng.choice(n, 24, replace=False))
    els = elements_touching(disc.mesh, dofs)
    xm = np.where(disc.mask, 0.0, x)
    Ue, Xe = disc.gather(u, els), disc.gather(xm, els)
    Ye = disc.ref.tangent_action(Ue, Xe, disc.mu, disc.lam) + b1 * disc.ref.mass_action(Xe, disc.rho)
    want = disc.scatter(Ye, els)[dofs]
    want = np.where(disc.mask[dofs], x[dofs], want)
    tol = TOL64 if prec == 0 else TOL32
    assert _relerr(yg[dofs], want) < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_forcing_terms_reach_the_same_state(prec):
    # Eisenstat-Walker forcing changes only the inner PCG tolerances; the
    # Newton test (1e-10 here) decides the state
    s = _sdme()
    w = workload("cube_p4")
    out = []
    for forcing in (0, 1):
        ctx, disc = _pair(elems=(2, 2, 2), lengths=(1.0, 1.0, 1.0), clamp={"zmin": (0, 1, 2)}, P=3, kind="sdme_h",
                          prec=prec, E=w["E"], nu=w["nu"], rho=w["rho"])
        f = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
        ctx.traction_load("zmax", (0.0, 0.0, -load_magnitude(w["load_key"])), f)
        u, v, a = (torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda") for _ in range(3))
        its = 0
        for n in range(1, 4):
            st = ctx.implicit_newmark_step(u, v, a, w["dt"], f * (n / 3.0), newton_tol=1e-10, forcing=forcing)
            assert st["converged"]
            its += st["pcg_iters_total"]
        out.append((_host(u), its))
    assert _relerr(out[1][0], out[0][0]) < 1e-8
    assert out[1][1] < out[0][1]
