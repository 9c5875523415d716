"""Write tests/golden/loads.json: traction magnitudes for the synthetic workloads.

Calls only the oracle.  Run from the repository root:

    python tests/golden/make_golden.py

* cube_p4_traction: dead uniform traction t_z = -s on the top face of the unit
  cube (bottom face clamped, E = 1000, nu = 0.3) such that the static mean top
  displacement is -0.10 (10% compressive strain).  Calibrated by secant
  iteration on the oracle at P = 3 on the same 4x4x4 mesh.
* beam_traction: dead shear traction t_z = -s on the x = 8 end of the
  [0,8]x[0,1]^2 cantilever (x = 0 clamped, E = 1000, nu = 0.45) such that the
  static mean tip deflection is -3.2 (40% of the length).  Calibrated by
  secant iteration on the oracle at P = 3 on a 16x2x2 mesh with 8 load
  increments per solve.

The face mean of u_z is (f . u) / A with f the load vector of a unit
traction (so f . u is the integral of u_z over the face, for any basis) and
A the face's area.  (The sum of f's entries equals A only for bases whose
functions sum to one: the Lagrange basis, not the modal or SDME ones.)
Linear solves: scipy's sparse LU of the assembled tangent.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import solvers  # noqa: E402
from oracle.assembly import Discretization  # noqa: E402
from oracle.basis1d import Basis1D  # noqa: E402
from oracle.hexmesh import BoxMesh  # noqa: E402
from oracle.material import lame  # noqa: E402


def _face_mean(disc, u, face, comp):
    """Area mean of u_comp over a face: traction load of a unit uniform
    traction dotted with u, divided by the face area."""
    t = np.zeros(3)
    t[comp] = 1.0
    f = disc.traction_load(face, lambda X, tt: np.broadcast_to(t, X.shape))
    axis = "xyz".index(face[0])
    L = disc.mesh.lengths
    area = float(np.prod([L[d] for d in range(3) if d != axis]))
    return float(f @ u) / area


def _static_response(disc, face, comp, s, nsteps):
    t = np.zeros(3)
    t[comp] = -1.0
    unit = disc.traction_load(face, lambda X, tt: np.broadcast_to(t, X.shape))
    u = np.zeros(disc.mesh.ndof)
    for k in range(1, nsteps + 1):
        u, st = solvers.static_newton(disc, unit * s * k / nsteps, u0=u, tol=1e-10, linear="sparse")
        if not st["converged"]:
            raise RuntimeError("static solve failed")
    return _face_mean(disc, u, face, comp)


def _secant(fun, target, s0, s1, tol=1e-6):
    f0, f1 = fun(s0) - target, fun(s1) - target
    for _ in range(30):
        s2 = s1 - f1 * (s1 - s0) / (f1 - f0)
        s0, f0 = s1, f1
        s1, f1 = s2, fun(s2) - target
        if abs(f1) < tol * abs(target):
            return s1
    raise RuntimeError("secant did not converge")


def main():
    out = {}
    mu, lam = lame(1000.0, 0.3)
    disc = Discretization(BoxMesh(4, 4, 4, 3).clamp("zmin"), Basis1D(3, "modal"), mu, lam)
    s = _secant(lambda s: _static_response(disc, "zmax", 2, s, 4), -0.10, 50.0, 100.0)
    out["cube_p4_traction"] = {"value": s, "how": "oracle, P=3, 4x4x4, static mean top u_z = -0.10"}
    print("cube", s)

    mu, lam = lame(1000.0, 0.45)
    disc = Discretization(BoxMesh(16, 2, 2, 3, (8.0, 1.0, 1.0)).clamp("xmin"), Basis1D(3, "modal"),
                          mu, lam)
    s = _secant(lambda s: _static_response(disc, "xmax", 2, s, 8), -3.2, 1.0, 1.6)
    out["beam_traction"] = {"value": s, "how": "oracle, P=3, 16x2x2, static mean tip u_z = -3.2"}
    print("beam", s)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "loads.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
