"""The headline path at reduced size: the cantilever of the benchmark
(x = 0 clamped, dead tip shear traction on x = 8 ramped over 20 implicit
Newmark steps of dt = 1, nu = 0.45, SDME-H) on 16x2x2 hexahedra at P = 2 and
8x1x1 at P = 4, through the C ABI in float64 and in mixed precision (float32
tangent and PCG with float64 refinement inside the float64 Newton residual),
against the oracle's Newmark steps (Sec. 4.2, eqs. Eq:residual and
NR_explicit) solved with dense direct linear solves.

Every step must converge on both sides (Newton test 1e-10 relative to
max(||psi_0||, ||P||), tighter than the benchmark's 1e-8), and the state
(u, v, a) must match the oracle's after every step: float64 1e-8, mixed
2e-8 relative in u (max-norm over the oracle's max-norm).  Both sides stop
at residuals <= 1e-10 of the load, so the states differ by at most that
residual through the inverse effective tangent; v and a inherit the
difference of u through the Newmark formulas (b1 = 4, b2 = 4 at dt = 1) and
are compared at 10x the tolerance of u.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import solvers  # noqa: E402
from oracle.assembly import Discretization  # noqa: E402
from oracle.basis1d import Basis1D  # noqa: E402
from oracle.hexmesh import BoxMesh  # noqa: E402
from oracle.material import lame  # noqa: E402
from synthetic import load_magnitude, workload  # noqa: E402

NEWTON_TOL = 1e-10
CASES = {"16x2x2_p2": ((16, 2, 2), 2), "8x1x1_p4": ((8, 1, 1), 4)}
_ORACLE = {}


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _oracle_ramp(case):
    """Oracle states after each of the 20 steps (computed once per case)."""
    if case in _ORACLE:
        return _ORACLE[case]
    w = workload("beam_p8")
    elems, P = CASES[case]
    mu, lam = lame(w["E"], w["nu"])
    mesh = BoxMesh(*elems, P, w["lengths"]).clamp("xmin")
    disc = Discretization(mesh, Basis1D(P, "sdme_h"), mu, lam, w["rho"])
    unit = disc.traction_load("xmax", lambda X, t: np.broadcast_to([0.0, 0.0, -1.0], X.shape))
    smag = load_magnitude(w["load_key"])
    u = np.zeros(mesh.ndof)
    v, a = u.copy(), u.copy()
    states = []
    for n in range(1, w["steps"] + 1):
        u, v, a, st = solvers.newmark_step(disc, u, v, a, unit * smag * n / w["steps"], w["dt"], tol=NEWTON_TOL,
                                           linear="direct")
        assert st["converged"], (case, n)
        states.append((u.copy(), v.copy(), a.copy()))
    _ORACLE[case] = (mesh.ndof, unit, states)
    return _ORACLE[case]


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cantilever_ramp_matches_oracle(case, prec):
    import paper_2104_13466_gb300 as s
    ndof, unit, states = _oracle_ramp(case)
    w = workload("beam_p8")
    elems, P = CASES[case]
    mu, lam = lame(w["E"], w["nu"])
    precision = s.MIXED_FP32 if prec == "mixed" else s.FP64
    ctx = s.Context(elems, w["lengths"], w["clamp"], mu, lam, w["rho"], P, "sdme_h", precision=precision)
    assert ctx.ndof == ndof
    f = torch.zeros(ndof, dtype=torch.float64, device="cuda")
    ctx.traction_load("xmax", (0.0, 0.0, -1.0), f)
    assert _relerr(f.cpu().numpy(), unit) < 1e-12
    smag = load_magnitude(w["load_key"])
    u, v, a = (torch.zeros(ndof, dtype=torch.float64, device="cuda") for _ in range(3))
    tol_u = 1e-8 if prec == "fp64" else 2e-8
    worst = 0.0
    for n in range(1, w["steps"] + 1):
        st = ctx.implicit_newmark_step(u, v, a, w["dt"], f * (smag * n / w["steps"]), newton_tol=NEWTON_TOL,
                                       pcg_rtol=1e-12, mixed_rtol=1e-4, max_newton=30, forcing=1)
        assert st["converged"] and st["residual_rel"] <= NEWTON_TOL, (n, st)
        uo, vo, ao = states[n - 1]
        torch.cuda.synchronize()
        eu = _relerr(u.cpu().numpy(), uo)
        ev = _relerr(v.cpu().numpy(), vo)
        ea = _relerr(a.cpu().numpy(), ao)
        worst = max(worst, eu)
        assert eu < tol_u and ev < 10 * tol_u and ea < 10 * tol_u, (n, eu, ev, ea)
    ctx.close()
