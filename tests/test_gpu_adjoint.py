"""GPU parity of the adjoint path against the oracle: the internal-force VJP
(K_T w and the (mu, lambda) partials), its torch.autograd wrapper, and the
checkpointed discrete adjoint of the explicit scheme (Sec. 4.1), plus the
gradient against central finite differences of the GPU forward.

Float64 throughout: VJP 1e-10 relative.  The trajectory adjoint differs from
the oracle's (direct mass solves) by the PCG mass-solve tolerance (1e-13)
amplified over the steps; bound 1e-8.  Finite differences (h = 1e-6
relative, central): 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adjoint  # noqa: E402
from oracle.assembly import Discretization  # noqa: E402
from oracle.basis1d import Basis1D  # noqa: E402
from oracle.hexmesh import BoxMesh  # noqa: E402
from oracle.material import lame  # noqa: E402

MU, LAM = lame(1000.0, 0.3)
TOL64 = 1e-10


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _pair(P, kind, elems=(2, 2, 1), prec=0, clamp=None):
    import paper_2104_13466_gb300 as s
    clamp = {"xmin": (0, 1, 2)} if clamp is None else clamp
    ctx = s.Context(elems, (1.0, 1.0, 1.0), clamp, MU, LAM, 1.0, P, kind, precision=prec)
    mesh = BoxMesh(*elems, P)
    for f, c in clamp.items():
        mesh.clamp(f, c)
    return ctx, Discretization(mesh, Basis1D(P, kind), MU, LAM, 1.0)


@pytest.mark.parametrize("P,kind", [(1, "nodal"), (2, "sdme_h"), (3, "nodal"), (4, "modal"), (5, "sdme_m"),
                                    (6, "sdme_k"), (8, "sdme_h")])
def test_vjp_matches_oracle(P, kind):
    ctx, d = _pair(P, kind, elems=(2, 1, 1) if P >= 6 else (3, 2, 2))
    rng = np.random.default_rng(P)
    u = 0.005 * rng.standard_normal(d.mesh.ndof)
    w = rng.standard_normal(d.mesh.ndof)
    gu = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    gmu, glam = ctx.internal_force_vjp(_dev(u), _dev(w), gu)
    gu_o, gmu_o, glam_o = adjoint.internal_force_vjp(d, u, w)
    assert _rel(_host(gu), gu_o) < TOL64
    assert abs(gmu - gmu_o) < TOL64 * abs(gmu_o) and abs(glam - glam_o) < TOL64 * abs(glam_o)


def test_vjp_in_mixed_context_is_float64():
    import paper_2104_13466_gb300 as s
    ctx, d = _pair(3, "sdme_h", prec=s.MIXED_FP32)
    rng = np.random.default_rng(1)
    u = 0.005 * rng.standard_normal(d.mesh.ndof)
    w = rng.standard_normal(d.mesh.ndof)
    gu = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    gmu, glam = ctx.internal_force_vjp(_dev(u), _dev(w), gu)
    gu_o, gmu_o, glam_o = adjoint.internal_force_vjp(d, u, w)
    assert _rel(_host(gu), gu_o) < TOL64 and abs(gmu - gmu_o) < TOL64 * abs(gmu_o)


def test_set_material_changes_forces_and_graph():
    ctx, d = _pair(2, "sdme_h")
    rng = np.random.default_rng(2)
    u = 0.005 * rng.standard_normal(d.mesh.ndof)
    R = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    ctx.set_material(2 * MU, 0.5 * LAM)
    ctx.internal_force(_dev(u), R)
    want = adjoint.internal_force_with(d, u, 2 * MU, 0.5 * LAM)
    assert _rel(_host(R), want) < TOL64
    # a PCG solve after the change uses the new material (graph re-captured)
    b = _dev(rng.standard_normal(d.mesh.ndof))
    x = torch.zeros_like(b)
    ctx.pcg_solve(_dev(u), 0.0, b, x, rtol=1e-12)
    d2 = Discretization(d.mesh, d.basis, 2 * MU, 0.5 * LAM, 1.0)
    r = d2.effective_apply(u, _host(x)) - np.where(d.mask, 0.0, _host(b))
    assert np.abs(r[~d.mask]).max() < 1e-9 * np.abs(_host(b)).max()


def test_invalid_material_rejected():
    import paper_2104_13466_gb300 as s
    ctx, _ = _pair(2, "sdme_h")
    with pytest.raises(s.SdmeError):
        ctx.set_material(-1.0, LAM)
    assert ctx.material[0] == MU


def test_autograd_internal_force():
    import paper_2104_13466_gb300 as s
    ctx, d = _pair(3, "sdme_m")
    rng = np.random.default_rng(3)
    u = _dev(0.005 * rng.standard_normal(d.mesh.ndof)).requires_grad_(True)
    w = _dev(rng.standard_normal(d.mesh.ndof))
    mu = torch.tensor(MU, dtype=torch.float64, requires_grad=True)
    lam = torch.tensor(LAM, dtype=torch.float64, requires_grad=True)
    loss = (s.internal_force(ctx, u, mu, lam) * w).sum()
    loss.backward()
    gu_o, gmu_o, glam_o = adjoint.internal_force_vjp(d, _host(u), _host(w))
    assert _rel(_host(u.grad), gu_o) < TOL64
    assert abs(mu.grad.item() - gmu_o) < TOL64 * abs(gmu_o)
    assert abs(lam.grad.item() - glam_o) < TOL64 * abs(glam_o)


def _trajectory_problem(d, seed=0, N=12):
    rng = np.random.default_rng(seed)
    n = d.mesh.ndof
    v0 = np.where(d.mask, 0.0, 0.05 * rng.standard_normal(n))
    f = 0.1 * rng.standard_normal(n)
    s = np.linspace(0.5, 1.0, N)
    target = 0.01 * rng.standard_normal(n)
    return v0, f, s, target


@pytest.mark.parametrize("every", [1, 5, 12])
def test_trajectory_adjoint_matches_oracle(every):
    import paper_2104_13466_gb300 as s
    ctx, d = _pair(3, "sdme_m")
    N, dt = 12, 1e-3
    v0, f, sch, target = _trajectory_problem(d, N=N)
    n = d.mesh.ndof
    u0 = np.zeros(n)
    traj = adjoint.explicit_run(d, u0, v0, f, sch, dt)
    g_o = adjoint.explicit_adjoint(d, traj, 2.0 * (traj[-1] - target), f, sch, dt)
    tape = s.Tape(ctx, N, every)
    uN = torch.zeros(n, dtype=torch.float64, device="cuda")
    tape.forward(dt, _dev(u0), _dev(v0), uN, f=_dev(f), s=sch, rtol=1e-14)
    assert _rel(_host(uN), traj[-1]) < 1e-10
    gN = _dev(2.0 * (_host(uN) - target))
    gu0, gv0, gf = (torch.zeros_like(gN) for _ in range(3))
    gmu, glam = tape.adjoint(gN, gu0, gv0, gf)
    assert abs(gmu - g_o["mu"]) < 1e-8 * abs(g_o["mu"])
    assert abs(glam - g_o["lam"]) < 1e-8 * abs(g_o["lam"])
    for name, t in (("u0", gu0), ("v0", gv0), ("f", gf)):
        assert _rel(_host(t), g_o[name]) < 1e-8, name
    tape.close()


def test_trajectory_autograd_and_finite_differences():
    import paper_2104_13466_gb300 as s
    ctx, d = _pair(2, "sdme_m", elems=(4, 1, 1), clamp={"xmin": (0, 1, 2)})
    N, dt = 20, 1e-3
    v0, f, sch, target = _trajectory_problem(d, seed=1, N=N)
    tape = s.Tape(ctx, N, 6)
    u0 = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    v0t, ft, tgt = _dev(v0), _dev(f), _dev(target)

    def J(mu, lam):
        uN = s.explicit_trajectory(tape, dt, u0, v0t, mu, lam, f=ft, s=sch, rtol=1e-14)
        return ((uN - tgt) ** 2).sum()

    mu = torch.tensor(MU, dtype=torch.float64, requires_grad=True)
    lam = torch.tensor(LAM, dtype=torch.float64, requires_grad=True)
    J(mu, lam).backward()
    with torch.no_grad():
        hm, hl = 1e-6 * MU, 1e-6 * LAM
        fd_mu = (J(MU + hm, LAM) - J(MU - hm, LAM)).item() / (2 * hm)
        fd_lam = (J(MU, LAM + hl) - J(MU, LAM - hl)).item() / (2 * hl)
    assert abs(mu.grad.item() - fd_mu) < 1e-5 * abs(fd_mu)
    assert abs(lam.grad.item() - fd_lam) < 1e-5 * abs(fd_lam)
    tape.close()
