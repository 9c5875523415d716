"""Pins for the oracle's static condensation (Schur complement on the
element-interior modes, Sec. 4 / Sec. 5.1).  CPU only."""
import json
import os

import numpy as np
import pytest

from oracle import condensation, manufactured, solvers
from oracle.assembly import Discretization
from oracle.basis1d import Basis1D
from oracle.hexmesh import BoxMesh
from oracle.material import lame

MU, LAM = lame(1000.0, 0.3)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _static(P, kind):
    d = Discretization(BoxMesh(2, 2, 2, P).clamp("xmin"), Basis1D(P, kind), MU, LAM)
    return d, manufactured.load_vector(d, manufactured.static_field(), 0.0)


@pytest.mark.parametrize("kind", ["modal", "sdme_h", "nodal"])
def test_condensed_solution_equals_direct(kind):
    d, f = _static(3, kind)
    u = 0.01 * np.random.default_rng(2).standard_normal(d.mesh.ndof)
    u[d.mask] = 0.0
    x, its = condensation.condensed_solve(d, u, f, b1=50.0, rtol=1e-13)
    xd = solvers.dense_solve(d.tangent_matrix(u, 50.0), np.where(d.mask, 0.0, f))
    assert np.abs(x - xd).max() < 1e-9 * np.abs(xd).max()
    assert its > 0


def test_interior_count_matches_paper_condensed_dofs():
    # the transient tables print condensed DOF counts: 276 at P = 2, 3084 at P = 6
    for P, want in ((2, 276), (6, 3084)):
        d = Discretization(BoxMesh(2, 2, 2, P).clamp("xmin"), Basis1D(P, "sdme_m"), MU, LAM)
        assert int((~d.mask & ~condensation.interior_mask(d.mesh)).sum()) == want


@pytest.mark.parametrize("P", [2, 4])
def test_condensed_cg_iterations_match_paper_static_table(P):
    with open(os.path.join(GOLDEN, "static_cgd_iterations.json")) as fh:
        g = json.load(fh)
    row = {r[0]: r[1:] for r in g["rows"]}[P]
    got = []
    for kind in ("modal", "sdme_m", "sdme_h"):
        d, f = _static(P, kind)
        u, st = condensation.static_newton_condensed(d, f, tol=1e-8, cg_rtol=1e-12)
        assert st["converged"] and st["newton_iters"] == 5
        got.append(np.mean(st["cg_iters"]))
    # average CGD iterations per Newton iteration within 15 % of the printed ones
    for have, want in zip(got, row):
        assert abs(have - want) < 0.15 * want, (got, row)
    # the ordering the paper reports: ST >> SDME-M >= SDME-H
    assert got[0] > 1.5 * got[1] and got[1] >= got[2]


def _newmark_condensed_iterations(P, kind, dt, T):
    d = Discretization(BoxMesh(2, 2, 2, P).clamp("xmin"), Basis1D(P, kind), MU, LAM)
    fld = manufactured.sine_field()
    u = np.zeros(d.mesh.ndof)
    v = d.l2_project(fld.velocity, 0.0)
    v[d.mask] = 0.0
    a = solvers.initial_acceleration(d, u, manufactured.load_vector(d, fld, 0.0))
    b1, b2, b3 = 4.0 / dt ** 2, 4.0 / dt, 1.0
    its = []
    for n in range(int(round(T / dt))):
        Pn = manufactured.load_vector(d, fld, (n + 1) * dt)
        const = b2 * v + b3 * a
        uk, psi0 = u.copy(), None
        for k in range(30):
            psi = Pn - d.mass_apply(b1 * (uk - u) - const) - d.internal_force(uk)
            psi[d.mask] = 0.0
            nrm = np.linalg.norm(psi)
            psi0 = nrm if psi0 is None else psi0
            if nrm <= 1e-12 * max(psi0, np.linalg.norm(Pn)):
                break
            du, it = condensation.condensed_solve(d, uk, psi, b1, 1e-12)
            its.append(it)
            uk = uk + du
        a_new = b1 * (uk - u) - const
        v = v + 0.5 * dt * (a + a_new)
        a, u = a_new, uk
    return np.mean(its)


def test_condensed_newmark_iterations_match_paper_table():
    with open(os.path.join(GOLDEN, "newmark_cgd_iterations.json")) as fh:
        g = json.load(fh)
    row = {r[0]: r[1:] for r in g["rows"]}[2]
    got = [_newmark_condensed_iterations(2, kind, g["dt"], g["T"]) for kind in ("modal", "sdme_m", "sdme_h")]
    for have, want in zip(got, row):
        assert abs(have - want) < 0.15 * want, (got, row)
    assert got[0] > 4 * got[1]
