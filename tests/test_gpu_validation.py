"""End-to-end validation on the GPU against the numbers the paper prints.

The product solves the paper's fabricated-solution problems (loads are
computed by the oracle from the closed-form fields, as test input) and the
oracle measures the L2 error of the GPU solution.  Checked against:

* Sec. 5.1, Table Static_error (static, 2x2x2 hexes, u_x = 1.9 sin x - x):
  same order-of-magnitude pin as the oracle's own test, the 5 Newton
  iterations of the paper, basis independence of the converged field, and
  parity with the oracle's static Newton solution;
* Sec. 5.2.1, Tables Transient_NH_L2errorHexa_SDME_M and
  Transient_NH_L2errorHexa_Lagrange (explicit, 800 steps): the SDME-M
  consistent-mass and the lumped-Lagrange variants.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import manufactured, solvers  # noqa: E402
from oracle.assembly import Discretization  # noqa: E402
from oracle.basis1d import Basis1D  # noqa: E402
from oracle.hexmesh import BoxMesh  # noqa: E402
from oracle.material import lame  # noqa: E402

MU, LAM = lame(1000.0, 0.3)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def _setup(P, kind, mass_rule="gauss"):
    import paper_2104_13466_gb300 as s
    ctx = s.Context((2, 2, 2), (1.0, 1.0, 1.0), {"xmin": (0, 1, 2)}, MU, LAM, 1.0, P, kind)
    okind = "nodal" if kind == "nodal_lumped" else kind
    d = Discretization(BoxMesh(2, 2, 2, P).clamp("xmin"), Basis1D(P, okind), MU, LAM, mass_rule=mass_rule)
    return ctx, d


@pytest.mark.parametrize("P", [2, 4, 6, 8])
def test_static_fabricated_table_on_gpu(P):
    g = _golden("static_fab_l2.json")
    row = [r for r in g["rows"] if r[0] == P][0]
    errs = []
    for kind in ("modal", "sdme_m", "sdme_h"):
        ctx, d = _setup(P, kind)
        fld = manufactured.static_field()
        f = manufactured.load_vector(d, fld, 0.0)
        u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
        st = ctx.static_solve(u, _dev(f), newton_tol=1e-8, pcg_rtol=1e-12)
        assert st["converged"] and st["newton_iters"] == g["newton_iterations"], st
        assert int((~d.mask).sum()) == row[1]
        err = d.l2_error(_host(u), fld.displacement)
        for have, want in zip(err, row[2:]):
            if P <= 4:
                assert want / 3.0 < have < want * 3.0, (kind, err, row)
            else:
                # the paper's volume rule is unstated; with Q = P + 2 Gauss
                # points the errors at P = 6, 8 come out below the printed
                # ones (P = 6: 3.6e-10 vs 4.5e-9), so only "no worse" is pinned
                assert have < want * 3.0, (kind, err, row)
        errs.append(err)
        if P <= 4:
            uo, so = solvers.static_newton(d, f, linear="direct")
            assert np.abs(_host(u) - uo).max() < 1e-9 * np.abs(uo).max()
    # "identical for all employed bases" (to the Newton tolerance's effect)
    assert np.allclose(errs[0], errs[1], rtol=1e-3) and np.allclose(errs[0], errs[2], rtol=1e-3)


def _explicit_fabricated(ctx, d, T, N, rtol):
    fld = manufactured.sine_field()
    dt = T / N
    n = d.mesh.ndof
    v0 = d.l2_project(fld.velocity, 0.0)
    v0[d.mask] = 0.0
    st = ctx.explicit_state(_dev(np.zeros(n)), _dev(np.zeros(n)), _dev(np.zeros(n)))
    ctx.explicit_start(st, dt, _dev(manufactured.load_vector(d, fld, 0.0)), _dev(v0), rtol=rtol)
    for k in range(N):
        ctx.explicit_step(st, dt, _dev(manufactured.load_vector(d, fld, k * dt)), rtol=rtol)
    return d.l2_error(_host(st.u), fld.displacement, T)


@pytest.mark.parametrize("kind,table", [("sdme_m", "explicit_fab_l2.json"),
                                        ("nodal_lumped", "explicit_fab_lagrange_l2.json")])
def test_explicit_fabricated_tables_on_gpu(kind, table):
    g = _golden(table)
    P = 2
    row = [r for r in g["rows"] if r[0] == P][0]
    ctx, d = _setup(P, kind, mass_rule="gll" if kind == "nodal_lumped" else "gauss")
    err = _explicit_fabricated(ctx, d, g["T"], g["steps"], rtol=1e-12)
    for have, want in zip(err, row[1:]):
        assert want / 3.0 < have < want * 3.0, (kind, err, row)


def _newmark_gpu(ctx, d, fld, dt, N, newton_tol=1e-11, pcg_rtol=1e-13):
    n = d.mesh.ndof
    v0 = d.l2_project(fld.velocity, 0.0)
    v0[d.mask] = 0.0
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    v = _dev(v0)
    # a_0 = M^{-1} (P_0 - R(u_0)) on the GPU
    R = torch.zeros_like(u)
    ctx.internal_force(u, R)
    a = torch.zeros_like(u)
    ctx.mass_solve(_dev(manufactured.load_vector(d, fld, 0.0)) - R, a, rtol=1e-14)
    stats = []
    for k in range(N):
        st = ctx.implicit_newmark_step(u, v, a, dt, _dev(manufactured.load_vector(d, fld, (k + 1) * dt)),
                                       newton_tol=newton_tol, pcg_rtol=pcg_rtol)
        assert st["converged"]
        stats.append(st)
    return _host(u), stats


def test_newmark_fabricated_table_on_gpu():
    g = _golden("newmark_fab_l2.json")
    P = 2
    row = [r for r in g["rows"] if r[0] == P][0]
    ctx, d = _setup(P, "sdme_h")
    fld = manufactured.sine_field()
    N = int(round(g["T"] / g["dt"]))
    u, stats = _newmark_gpu(ctx, d, fld, g["dt"], N)
    # the transient tables count the statically condensed (skeleton) DOFs:
    # free DOFs minus the 3 (P - 1)^3 internal ones of each element
    assert int((~d.mask).sum()) - 3 * (P - 1) ** 3 * d.mesh.nelem == row[1]
    err = d.l2_error(u, fld.displacement, g["T"])
    for have, want in zip(err, row[2:]):
        assert want / 3.0 < have < want * 3.0, (err, row)


def test_newmark_second_order_in_time_on_gpu():
    # Sec. 5.2.2: u_x = x^4 sin(2 pi t) is represented exactly in space at
    # P = 5, so the error at T = 0.025 is the time error; halving dt must
    # divide it by ~4 (quadratic rate of the Newmark scheme)
    P, T = 5, 0.025
    ctx, d = _setup(P, "sdme_h")
    fld = manufactured.quartic_field()
    errs = []
    for N in (4, 8, 16):
        u, _ = _newmark_gpu(ctx, d, fld, T / N, N, newton_tol=1e-12, pcg_rtol=1e-14)
        errs.append(d.l2_error(u, fld.displacement, T)[0])
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < r < 2.2 for r in rates), (errs, rates)
