"""GPU parity of the plane-strain quadrilateral path (eq. ProdTensorialQuadrado)
against the oracle's 2D discretisation (itself pinned to the 3D one).
Float64 1e-10 relative; mixed-precision operators 2e-5."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import quad, solvers  # noqa: E402
from oracle.basis1d import Basis1D  # noqa: E402
from oracle.material import lame  # noqa: E402

MU, LAM = lame(1000.0, 0.3)
TOL64, TOL32 = 1e-10, 2e-5


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _pair(P, kind, elems=(3, 2), lengths=(1.5, 1.0), clamp=None, prec=0, rho=1.2):
    import paper_2104_13466_gb300 as s
    clamp = {"xmin": (0, 1)} if clamp is None else clamp
    ctx = s.Context(elems, lengths, clamp, MU, LAM, rho, P, kind, precision=prec)
    mesh = quad.RectMesh(*elems, P, lengths=lengths)
    for f, c in clamp.items():
        mesh.clamp(f, c)
    return ctx, quad.Discretization2D(mesh, Basis1D(P, kind), MU, LAM, rho)


def _u(d, seed, amp=0.01):
    h = min(d.mesh.h) / d.mesh.P
    return amp * h * np.random.default_rng(seed).standard_normal(d.mesh.ndof)


@pytest.mark.parametrize("P,kind", [(1, "nodal"), (2, "modal"), (3, "nodal"), (4, "sdme_h"), (5, "sdme_m"),
                                    (6, "sdme_k"), (7, "modal"), (8, "sdme_h")])
def test_quad_operators_fp64(P, kind):
    ctx, d = _pair(P, kind)
    assert ctx.ndof == d.mesh.ndof
    u = _u(d, P)
    x = np.random.default_rng(P + 10).standard_normal(d.mesh.ndof)
    R = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.internal_force(_dev(u), R)
    assert _rel(_host(R), d.internal_force(u)) < TOL64
    y = torch.zeros_like(R)
    ctx.tangent_apply(_dev(u), 30.0, _dev(x), y)
    assert _rel(_host(y), d.effective_apply(u, x, b1=30.0)) < TOL64
    dg = torch.zeros_like(R)
    ctx.diagonal(_dev(u), 30.0, dg)
    assert _rel(_host(dg), d.diagonal(u, 30.0)) < TOL64
    m = torch.zeros_like(R)
    ctx.mass_apply(_dev(x), m)
    assert _rel(_host(m), d.mass_apply(x)) < TOL64
    ke, se = ctx.energy(_dev(u), _dev(x))
    assert abs(se - d.energy(u)) < 1e-10 * abs(d.energy(u))
    assert abs(ke - d.kinetic_energy(x)) < 1e-11 * abs(d.kinetic_energy(x))


def test_quad_tangent_mixed():
    import paper_2104_13466_gb300 as s
    ctx, d = _pair(4, "sdme_h", prec=s.MIXED_FP32)
    u = _u(d, 3)
    x = np.random.default_rng(4).standard_normal(d.mesh.ndof)
    y = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.tangent_apply(_dev(u), 10.0, _dev(x), y)
    assert _rel(_host(y), d.effective_apply(u, x, b1=10.0)) < TOL32


def test_quad_pcg_matches_dense():
    ctx, d = _pair(3, "sdme_m", elems=(2, 2))
    u = _u(d, 5)
    b = np.random.default_rng(6).standard_normal(d.mesh.ndof)
    x = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    its, rel = ctx.pcg_solve(_dev(u), 50.0, _dev(b), x, rtol=1e-13)
    xd = solvers.dense_solve(d.tangent_matrix(u, 50.0), np.where(d.mask, 0.0, b))
    assert _rel(_host(x), xd) < 1e-9 and its > 0


def test_quad_traction_and_newmark_steps():
    ctx, d = _pair(3, "sdme_h", elems=(3, 1), lengths=(3.0, 1.0))
    f = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.traction_load("xmax", (0.0, -20.0, 0.0), f)
    fo = d.traction_load("xmax", (0.0, -20.0))
    assert _rel(_host(f), fo) < 1e-13
    u, v, a = (torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda") for _ in range(3))
    uo, vo, ao = (np.zeros(d.mesh.ndof) for _ in range(3))
    for k in range(1, 4):
        st = ctx.implicit_newmark_step(u, v, a, 0.02, f * (k / 3.0), newton_tol=1e-12, pcg_rtol=1e-13)
        assert st["converged"]
        uo, vo, ao, so = solvers.newmark_step(d, uo, vo, ao, fo * (k / 3.0), 0.02, tol=1e-12, pcg_rtol=1e-13)
    assert _rel(_host(u), uo) < 1e-9 and _rel(_host(v), vo) < 1e-8


def test_quad_explicit_steps():
    ctx, d = _pair(4, "sdme_m", elems=(2, 2))
    n = d.mesh.ndof
    v0 = np.where(d.mask, 0.0, 0.01 * np.random.default_rng(7).standard_normal(n))
    f = np.zeros(n)
    dt = 1e-4
    st = ctx.explicit_state(_dev(np.zeros(n)), _dev(np.zeros(n)), _dev(np.zeros(n)))
    ctx.explicit_start(st, dt, _dev(f), _dev(v0), rtol=1e-14)
    up, _ = solvers.central_difference_start(d, np.zeros(n), v0, f, dt)
    u = np.zeros(n)
    Mm = solvers._masked_mass(d)
    for k in range(5):
        ctx.explicit_step(st, dt, _dev(f), rtol=1e-14)
        un, _ = solvers.central_difference_step(d, u, up, f, dt, Mm=Mm)
        up, u = u, un
    assert _rel(_host(st.u), u) < 1e-10


def test_quad_unsupported_operations():
    import paper_2104_13466_gb300 as s
    ctx, d = _pair(2, "sdme_h")
    z = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(s.SdmeError) as ei:
        ctx.internal_force_vjp(z, z, z.clone())
    assert ei.value.status == s.EUNSUPPORTED
    with pytest.raises(s.SdmeError):
        ctx.set_condensation(True)
