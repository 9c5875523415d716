"""Adjoints of the internal force and of the explicit scheme (oracle; test
infrastructure only).

The paper has no adjoint; these are the exact derivatives of what it
defines, written from the definitions:

* ``internal_force_vjp``: for R(u; mu, lambda) = sum_e int P(F) : grad N dV
  with P = mu (F - F^{-T}) + lambda ln J F^{-T} (Sec. 3),
  (dR/du)^T w = K_T(u) w because the consistent tangent is the Hessian of the
  strain energy (symmetric), and R is linear in (mu, lambda), so
  w . dR/dmu = w . R(u; 1, 0) and w . dR/dlambda = w . R(u; 0, 1).
* ``explicit_run`` / ``explicit_adjoint``: the central-difference scheme of
  Sec. 4.1 (start-up and eq. Motion_explicit2 as in ``solvers``) and its
  discrete adjoint, the transpose of each step's Jacobian applied in reverse
  step order.  The scheme's step maps (u_n, u_{n-1}) to
      u_{n+1} = 2 u_n - u_{n-1} + dt^2 A (P_n - R(u_n))   (free DOFs),
      u_{n+1} = u_n                                        (constrained DOFs),
  with A = M^{-1} on the free DOFs (zero rows/columns on constrained ones),
  and the start-up is u_{-1} = u_0 - dt v_0 + dt^2/2 A (P_0 - R(u_0)).

Pins (tests/test_oracle_adjoint.py): central finite differences of R and of
the whole trajectory objective with respect to u, mu, lambda, v_0, u_0 and
the load.
"""
import copy

import numpy as np

from . import solvers


def internal_force_with(disc, u, mu, lam):
    """R(u) with the material constants replaced by (mu, lam)."""
    d = copy.copy(disc)
    d.mu, d.lam = float(mu), float(lam)
    return d.internal_force(u)


def internal_force_vjp(disc, u, w):
    """((dR/du)^T w, w . dR/dmu, w . dR/dlambda), all DOFs, no Dirichlet treatment."""
    gu = disc.tangent_apply(u, w)
    gmu = float(w @ internal_force_with(disc, u, 1.0, 0.0))
    glam = float(w @ internal_force_with(disc, u, 0.0, 1.0))
    return gu, gmu, glam


def explicit_run(disc, u0, v0, f, s, dt):
    """Central-difference trajectory with loads P_n = s[n] f, n = 0 .. N-1
    (N = len(s)).  Returns the list [u_{-1}, u_0, u_1, ..., u_N]."""
    Mm = solvers._masked_mass(disc)
    up, _ = solvers.central_difference_start(disc, u0, v0, s[0] * f, dt)
    traj = [up, u0.copy()]
    u = u0.copy()
    for n in range(len(s)):
        un, _ = solvers.central_difference_step(disc, u, up, s[n] * f, dt, Mm=Mm)
        up, u = u, un
        traj.append(u)
    return traj


def explicit_adjoint(disc, traj, gN, f, s, dt):
    """Gradients of J(u_N) from gN = dJ/du_N for the trajectory of
    ``explicit_run``: returns dict with mu, lam, u0, v0, f."""
    N = len(s)
    free = ~disc.mask
    Mm = solvers._masked_mass(disc)

    def A(x):
        return solvers.mass_solve(disc, x, Mm=Mm)

    def u_at(n):
        return traj[n + 1]

    dt2 = dt * dt
    g1, g2 = gN.copy(), np.zeros_like(gN)      # g_{n+1}, g_{n+2}
    gmu = glam = 0.0
    gf = np.zeros_like(gN)
    for n in range(N - 1, -1, -1):
        z = A(g1)
        Kz, pm, pl = internal_force_vjp(disc, u_at(n), z)
        gmu -= dt2 * pm
        glam -= dt2 * pl
        gf += dt2 * s[n] * z
        gn = np.where(free, 2.0 * g1 - g2, g1) - dt2 * Kz
        g1, g2 = gn, g1
    # start-up: u_1 depends on u_{-1} through -u_{-1} on free DOFs
    g0, g1 = g1, g2
    gm1 = np.where(free, -g1, 0.0)
    z = A(gm1)
    Kz, pm, pl = internal_force_vjp(disc, u_at(0), z)
    gmu -= 0.5 * dt2 * pm
    glam -= 0.5 * dt2 * pl
    gf += 0.5 * dt2 * s[0] * z
    gu0 = g0 + gm1 - 0.5 * dt2 * Kz
    gv0 = -dt * gm1
    return {"mu": gmu, "lam": glam, "u0": gu0, "v0": gv0, "f": gf}
