"""Float64 refinement of the float32 PCG (SDME_MIXED_FP32).

A stiffness-dominated slender cantilever (b1 -> 0, nu = 0.45) is the case
where a float32 solve cannot meet a tight tolerance with respect to the
float64 operator: the float32 operator differs from the float64 one by about
eps32 times the element-level forces, far above the assembled forces of the
smooth bending modes the solution is made of.  With the refinement, the
solve's float64 residual b - (b1 M + K_T) x, recomputed here through a
float64 context, meets the tolerance, and the reported relative residual is
that float64 one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.material import lame  # noqa: E402


def _beam(prec):
    import paper_2104_13466_gb300 as s
    mu, lam = lame(1000.0, 0.45)
    return s.Context((32, 2, 2), (8.0, 1.0, 1.0), {"xmin": (0, 1, 2)}, mu, lam, 1.0, 4, "sdme_k", precision=prec)


def _true_rel(ctx64, b1, b, x):
    u = torch.zeros_like(b)
    y = torch.zeros_like(b)
    ctx64.tangent_apply(u, b1, x, y)
    free = torch.ones_like(b)
    free[:: ctx64.N[0]] = 0.0            # x = 0 face (ix = 0) is clamped
    return float(torch.linalg.norm((b - y) * free) / torch.linalg.norm(b * free))


def test_refined_float32_solve_meets_the_float64_tolerance():
    import paper_2104_13466_gb300 as s
    c32, c64 = _beam(s.MIXED_FP32), _beam(s.FP64)
    b = torch.zeros(c32.ndof, dtype=torch.float64, device="cuda")
    c32.traction_load("xmax", (0.0, 0.0, -1.0), b)
    b1, rtol = 1e-6, 1e-6
    u = torch.zeros_like(b)
    x = torch.zeros_like(b)
    its, rel = c32.pcg_solve(u, b1, b, x, rtol=rtol, maxit=200000)
    true = _true_rel(c64, b1, b, x)
    assert rel <= rtol and true <= 1.05 * rtol, (rel, true)
    assert abs(true - rel) <= 1e-3 * rtol + 1e-2 * rel, (rel, true)
    # the same solve without refinement stops on the float32 recurrence's own
    # test; its float64 residual is far above the tolerance
    c32.set_refinement(0)
    x0 = torch.zeros_like(b)
    c32.pcg_solve(u, b1, b, x0, rtol=rtol, maxit=200000)
    assert _true_rel(c64, b1, b, x0) > 10 * true
    c32.close()
    c64.close()


def test_refinement_count_is_validated():
    import paper_2104_13466_gb300 as s
    c = _beam(s.MIXED_FP32)
    with pytest.raises(s.SdmeError):
        c.set_refinement(-1)
    c.close()
