"""Pins for the oracle's adjoints (internal-force VJP and the discrete adjoint
of the explicit scheme, Sec. 4.1) by central finite differences.  CPU only."""
import numpy as np
import pytest

from oracle import adjoint
from oracle.assembly import Discretization
from oracle.basis1d import Basis1D
from oracle.hexmesh import BoxMesh
from oracle.material import lame

MU, LAM = lame(1000.0, 0.3)


def _disc(P=2, kind="sdme_h", elems=(2, 1, 1), mu=MU, lam=LAM):
    return Discretization(BoxMesh(*elems, P).clamp("xmin"), Basis1D(P, kind), mu, lam)


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("kind", ["nodal", "sdme_h"])
def test_internal_force_vjp_matches_finite_differences(kind):
    d = _disc(kind=kind)
    rng = np.random.default_rng(3)
    n = d.mesh.ndof
    u = 0.05 * rng.standard_normal(n)
    w = rng.standard_normal(n)
    v = rng.standard_normal(n)
    gu, gmu, glam = adjoint.internal_force_vjp(d, u, w)
    h = 1e-6
    fd_u = (w @ d.internal_force(u + h * v) - w @ d.internal_force(u - h * v)) / (2 * h)
    assert _rel(gu @ v, fd_u) < 1e-7
    hm = 1e-6 * MU
    fd_mu = (w @ adjoint.internal_force_with(d, u, MU + hm, LAM)
             - w @ adjoint.internal_force_with(d, u, MU - hm, LAM)) / (2 * hm)
    hl = 1e-6 * LAM
    fd_lam = (w @ adjoint.internal_force_with(d, u, MU, LAM + hl)
              - w @ adjoint.internal_force_with(d, u, MU, LAM - hl)) / (2 * hl)
    assert _rel(gmu, fd_mu) < 1e-7 and _rel(glam, fd_lam) < 1e-7
    # linearity in (mu, lambda): R = mu R_mu + lambda R_lambda
    assert _rel(MU * gmu + LAM * glam, w @ d.internal_force(u)) < 1e-12


def test_internal_force_vjp_zero_at_rest():
    d = _disc()
    w = np.random.default_rng(4).standard_normal(d.mesh.ndof)
    gu, gmu, glam = adjoint.internal_force_vjp(d, np.zeros(d.mesh.ndof), w)
    assert gmu == pytest.approx(0.0, abs=1e-12) and glam == pytest.approx(0.0, abs=1e-12)
    # at u = 0 the tangent is the linear-elastic stiffness: symmetric
    v = np.random.default_rng(5).standard_normal(d.mesh.ndof)
    assert _rel(v @ gu, w @ d.tangent_apply(np.zeros(d.mesh.ndof), v)) < 1e-12


def _problem(seed=0, N=6, P=2):
    d = _disc(P=P, kind="sdme_m")
    rng = np.random.default_rng(seed)
    n = d.mesh.ndof
    v0 = np.where(d.mask, 0.0, 0.5 * rng.standard_normal(n))
    f = 10.0 * rng.standard_normal(n)
    s = np.linspace(0.5, 1.0, N)
    target = 0.01 * rng.standard_normal(n)
    return d, v0, f, s, target


def _objective(d, u0, v0, f, s, dt, target):
    uN = adjoint.explicit_run(d, u0, v0, f, s, dt)[-1]
    return float(np.sum((uN - target) ** 2)), uN


def test_explicit_adjoint_matches_finite_differences():
    d, v0, f, s, target = _problem()
    dt = 2e-3
    n = d.mesh.ndof
    u0 = np.zeros(n)
    traj = adjoint.explicit_run(d, u0, v0, f, s, dt)
    g = adjoint.explicit_adjoint(d, traj, 2.0 * (traj[-1] - target), f, s, dt)

    def J(dd=d, uu=u0, vv=v0, ff=f):
        return _objective(dd, uu, vv, ff, s, dt, target)[0]

    for name, base in (("mu", MU), ("lam", LAM)):
        h = 1e-6 * base
        dp = _disc(kind="sdme_m", mu=MU + (h if name == "mu" else 0), lam=LAM + (h if name == "lam" else 0))
        dm = _disc(kind="sdme_m", mu=MU - (h if name == "mu" else 0), lam=LAM - (h if name == "lam" else 0))
        fd = (J(dd=dp) - J(dd=dm)) / (2 * h)
        assert _rel(g[name], fd) < 1e-6, (name, g[name], fd)
    rng = np.random.default_rng(9)
    for name in ("u0", "v0", "f"):
        p = rng.standard_normal(n)
        h = 1e-6
        if name == "u0":
            p = 1e-3 * p
            fd = (J(uu=u0 + h * p) - J(uu=u0 - h * p)) / (2 * h)
        elif name == "v0":
            fd = (J(vv=v0 + h * p) - J(vv=v0 - h * p)) / (2 * h)
        else:
            fd = (J(ff=f + h * p) - J(ff=f - h * p)) / (2 * h)
        assert _rel(g[name] @ p, fd) < 1e-6, (name, g[name] @ p, fd)


def test_explicit_adjoint_linear_limit():
    # a zero-amplitude trajectory is governed by the linear-elastic operator:
    # with u0 = v0 = f = 0 the state stays 0 and only the terminal adjoint
    # propagates; the material gradient is then exactly zero
    d, v0, f, s, target = _problem(N=4)
    n = d.mesh.ndof
    traj = adjoint.explicit_run(d, np.zeros(n), np.zeros(n), np.zeros(n), s, 1e-3)
    assert all(np.abs(t).max() == 0.0 for t in traj)
    g = adjoint.explicit_adjoint(d, traj, -2.0 * target, np.zeros(n), s, 1e-3)
    assert g["mu"] == 0.0 and g["lam"] == 0.0
