"""Seeded synthetic inputs shared by the oracle-side tests and the GPU path.

This module holds workload descriptions (mesh sizes, orders, material
constants, boundary faces, step sizes, seeds) and seeded random number draws
only.  It contains none of the method's arithmetic: no basis, quadrature,
material law or solver.  Both the oracle and the product turn these plain
numbers into their own data structures independently.

Workloads follow the paper's test shapes (Sec. 5: unit cubes of hexahedra,
neo-Hookean E = 1000, nu = 0.3, rho = 1; bases ST/nodal/SDME with k = 0.5 and
lambda = 100) scaled to the GPU problem sizes:

* ``cube_p4``   unit cube, 4x4x4 hexes, P = 4; bottom face clamped, uniform
                dead top traction ramped over 10 implicit Newmark steps.
* ``beam_p8``   [0,8]x[0,1]x[0,1] cantilever, 64x8x8 hexes, P = 8, nu = 0.45;
                x = 0 clamped, dead shear traction on x = 8 ramped over 20 steps.
* ``beam_p8_dyn``  the same cantilever with dt = 3e-4, the paper's ratio of
                time step to element wave-transit time (mass-dominated steps).
* ``cube_p6_explicit``  explicit central-difference run on the unit cube,
                16^3 hexes, P = 6 (2.74 M DOFs), all faces clamped, seeded
                sinusoidal initial velocity, 2000 steps at half the stable step.
* ``beam_p6_adjoint``  differentiated explicit run: [0,8]x[0,1]x[0,1]
                cantilever, 32x4x4 hexes, P = 6 (361,875 DOFs), x = 0 clamped,
                constant dead traction on x = 8, 200 steps at half the stable
                step, checkpoints every 20 steps; objective = squared distance of
                the final tip-face displacement to a seeded target.
* ``batch_cubes``  256 independent unit cubes: n^3 hexes with n ~ U{2..12},
                P uniform over {3, 4, 5, 6, 8}, E ~ U[5e2, 5e3], nu ~ U[0.25, 0.45]
                (all from `seed`); bottom face clamped, uniform top traction
                (half the cube_p4 magnitude, scaled by E / 1000) ramped over 20
                implicit Newmark steps, dt = 0.01.  At the full magnitude the
                finest nearly incompressible cube (12^3, P = 8, nu = 0.447)
                inverts elements at its clamped bottom edges during the ramp.
* ``static_fab``  the paper's static fabricated problem (Sec. 5.1): unit cube,
                2x2x2 hexes, x = 0 clamped.

Load magnitudes are produced by ``tests/golden/make_golden.py`` (which calls
only the oracle) and stored in ``tests/golden/loads.json``.
"""
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LOADS = os.path.join(os.path.dirname(_HERE), "tests", "golden", "loads.json")

WORKLOADS = {
    "cube_p4": dict(
        elems=(4, 4, 4), P=4, lengths=(1.0, 1.0, 1.0), E=1.0e3, nu=0.3, rho=1.0,
        clamp={"zmin": (0, 1, 2)}, traction_face="zmax", traction_dir=(0.0, 0.0, -1.0),
        steps=10, dt=0.01, newton_tol=1e-8, pcg_rtol=1e-10, k=0.5, lam=100.0,
        load_key="cube_p4_traction"),
    # basis: SDME-K, the lambda -> 0 limit of SDME-H; the Helmholtz
    # parameter tied to the Newmark coefficient in reference-element units,
    # lambda = b1 h^2 / (4 c^2) with c^2 = (lambda_L + 2 mu) / rho, is 4e-6 at
    # dt = 1 (stiffness-dominated steps)
    "beam_p8": dict(
        elems=(64, 8, 8), P=8, lengths=(8.0, 1.0, 1.0), E=1.0e3, nu=0.45, rho=1.0,
        clamp={"xmin": (0, 1, 2)}, traction_face="xmax", traction_dir=(0.0, 0.0, -1.0),
        steps=20, dt=1.0, newton_tol=1e-8, pcg_rtol=1e-10, k=0.5, lam=100.0,
        load_key="beam_traction", basis="sdme_k"),
    # the same cantilever in the paper's dynamic regime: dt = 0.15 h / c_L
    # (h = 0.125, c_L = sqrt((lambda + 2 mu) / rho) = 61.6 for nu = 0.45), the
    # ratio of the paper's implicit fabricated tests (dt = 2e-3, h = 0.5,
    # c_L = 36.7); the tip load is ramped over the same 20 steps
    "beam_p8_dyn": dict(
        elems=(64, 8, 8), P=8, lengths=(8.0, 1.0, 1.0), E=1.0e3, nu=0.45, rho=1.0,
        clamp={"xmin": (0, 1, 2)}, traction_face="xmax", traction_dir=(0.0, 0.0, -1.0),
        steps=20, dt=3.0e-4, newton_tol=1e-8, pcg_rtol=1e-10, k=0.5, lam=100.0,
        load_key="beam_traction"),
    # explicit elastodynamics: unit cube of 16^3 hexes at P = 6, all faces
    # clamped, initial velocity v_amp (1 + 0.01 xi) sin(pi x) sin(pi y)
    # sin(pi z) e_z with xi ~ U(-1, 1) drawn from `seed`, no load, steps at
    # cfl x the critical step
    "cube_p6_explicit": dict(
        elems=(16, 16, 16), P=6, lengths=(1.0, 1.0, 1.0), E=1.0e3, nu=0.3, rho=1.0,
        clamp={f: (0, 1, 2) for f in ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")},
        v_amp=0.05, seed=0, cfl=0.5, steps=2000, mass_rtol=1e-12, mass_rtol_mixed=1e-6),
    # objective target: tip-face lattice points, z-component
    # -tip_delta (1 + 0.1 xi), xi ~ U(-1, 1) from `seed`, x and y components 0
    "beam_p6_adjoint": dict(
        elems=(32, 4, 4), P=6, lengths=(8.0, 1.0, 1.0), E=1.0e3, nu=0.3, rho=1.0,
        clamp={"xmin": (0, 1, 2)}, traction_face="xmax", traction=(0.0, 0.0, -10.0),
        steps=200, every=20, cfl=0.5, seed=0, tip_delta=1e-3, mass_rtol=1e-12, fd_rel_h=1e-6),
    "batch_cubes": dict(
        count=256, side=(2, 12), orders=(3, 4, 5, 6, 8), E=(5.0e2, 5.0e3), nu=(0.25, 0.45), rho=1.0, seed=0,
        clamp={"zmin": (0, 1, 2)}, traction_face="zmax", steps=20, dt=0.01, newton_tol=1e-8, k=0.5, lam=100.0,
        load_key="cube_p4_traction", load_scale=0.5),
    "static_fab": dict(
        elems=(2, 2, 2), P=4, lengths=(1.0, 1.0, 1.0), E=1.0e3, nu=0.3, rho=1.0,
        clamp={"xmin": (0, 1, 2)}, k=0.5, lam=100.0),
}


def workload(name, **overrides):
    w = dict(WORKLOADS[name])
    w.update(overrides)
    return w


def load_magnitude(key):
    """Traction magnitude stored by the golden script (oracle calibration)."""
    with open(_LOADS) as f:
        return float(json.load(f)[key]["value"])


def rng(seed):
    return np.random.default_rng(seed)


def random_vector(n, seed, scale=1.0):
    """n standard-normal draws times ``scale`` (float64)."""
    return rng(seed).standard_normal(n) * scale


def random_uniform(n, seed, lo=-1.0, hi=1.0):
    return rng(seed).uniform(lo, hi, n)


def batch_draws(w):
    """Seeded per-problem draws of a batch workload: (side, P, E, nu) lists."""
    g = rng(w["seed"])
    n = w["count"]
    side = g.integers(w["side"][0], w["side"][1] + 1, n)
    P = g.choice(np.asarray(w["orders"]), n)
    E = g.uniform(w["E"][0], w["E"][1], n)
    nu = g.uniform(w["nu"][0], w["nu"][1], n)
    return [int(v) for v in side], [int(v) for v in P], [float(v) for v in E], [float(v) for v in nu]
