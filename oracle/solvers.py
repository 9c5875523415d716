"""Linear and nonlinear solvers (oracle; test infrastructure only).

* ``jacobi_pcg``: conjugate gradient with the diagonal (Jacobi) preconditioner,
  the paper's CGD / element-by-element diagonal PCG (Sec. 5, Conrod;
  conclusions).  Stopping rule (reading; the paper gives only tolerances):
  ||r||_2 <= rtol ||b||_2 on the unpreconditioned residual, x0 = 0.
* ``dense_solve`` / ``sparse_solve``: direct solve of the assembled system
  (dense LU for tiny meshes, scipy's sparse LU for small ones).
* ``newmark_step``: one implicit Newmark step solved by Newton-Raphson
  (Sec. 4.2, eqs. Eq:residual, NR_explicit).  The paper's coefficient table
  for the Newmark approximations is garbled; the reading is the standard
  Newmark family with beta = 0.25, gamma = 0.5:
      a_{n+1} = b1 (u_{n+1} - u_n) - b2 v_n - b3 a_n,
      b1 = 1/(beta dt^2), b2 = 1/(beta dt), b3 = (1 - 2 beta)/(2 beta),
      v_{n+1} = v_n + dt [(1 - gamma) a_n + gamma a_{n+1}].
  Predictor u^0_{n+1} = u_n (last converged step).  Newton stops when
  ||psi^k|| <= tol max(||psi^0||, ||P_{n+1}||): the paper gives the Newton
  tolerance (1e-8, Sec. 5.1) without its reference; it is read as relative
  to the larger of the step's initial residual and the applied load.
* ``static_newton``: the same Newton loop without inertia (Sec. 5.1).
"""
import numpy as np


def jacobi_pcg(apply, b, d, rtol=1e-10, maxit=10000):
    """Solve A x = b by diagonal-preconditioned CG; returns (x, iters, relres)."""
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    r = b.copy()
    z = r / d
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = apply(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        rn = np.linalg.norm(r)
        if rn <= rtol * bn:
            return x, it, rn / bn
        z = r / d
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, np.linalg.norm(r) / bn


def dense_solve(A, b):
    A = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    return np.linalg.solve(A, b)


def sparse_solve(A, b):
    """Direct solve of the assembled sparse system (scipy's sparse LU)."""
    import scipy.sparse.linalg as spla
    return spla.spsolve(A.tocsc(), b)


def _newton(disc, u, residual_fn, b1, tol, pcg_rtol, maxnewton, linear, pload_norm, stats):
    mask = disc.mask
    psi0 = None
    for k in range(maxnewton + 1):
        psi = residual_fn(u)
        psi[mask] = 0.0
        nrm = np.linalg.norm(psi)
        if psi0 is None:
            psi0 = nrm
        stats["residuals"].append(nrm)
        if nrm <= tol * max(psi0, pload_norm):
            stats["newton_iters"] = k
            return u, True
        if k == maxnewton:
            break
        if linear == "direct":
            du = dense_solve(disc.tangent_matrix(u, b1), psi)
            stats["pcg_iters"].append(0)
        elif linear == "sparse":
            du = sparse_solve(disc.tangent_matrix(u, b1), psi)
            stats["pcg_iters"].append(0)
        else:
            d = disc.diagonal(u, b1)
            du, its, _ = jacobi_pcg(lambda x: disc.effective_apply(u, x, b1), psi, d, pcg_rtol)
            stats["pcg_iters"].append(its)
        du[mask] = 0.0
        u = u + du
    stats["newton_iters"] = maxnewton
    return u, False


def newmark_step(disc, un, vn, an, Pnext, dt, beta=0.25, gamma=0.5, tol=1e-8,
                 pcg_rtol=1e-10, maxnewton=30, linear="pcg", u_pred=None):
    """One Newmark step (Sec. 4.2); returns (u, v, a, stats)."""
    b1 = 1.0 / (beta * dt * dt)
    b2 = 1.0 / (beta * dt)
    b3 = (1.0 - 2.0 * beta) / (2.0 * beta)
    const = b2 * vn + b3 * an

    def accel(u):
        return b1 * (u - un) - const

    def residual(u):
        # eq. NR_explicit right-hand side: -M a - R + P
        return Pnext - disc.internal_force(u) - disc.mass_apply(accel(u))

    stats = {"residuals": [], "pcg_iters": []}
    u0 = un.copy() if u_pred is None else u_pred.copy()
    u, ok = _newton(disc, u0, residual, b1, tol, pcg_rtol, maxnewton, linear,
                    np.linalg.norm(Pnext), stats)
    stats["converged"] = ok
    a = accel(u)
    v = vn + dt * ((1.0 - gamma) * an + gamma * a)
    return u, v, a, stats


def static_newton(disc, Pext, u0=None, tol=1e-8, pcg_rtol=1e-12, maxnewton=50, linear="pcg"):
    """Newton-Raphson for R(u) = P (Sec. 5.1 static problem)."""
    stats = {"residuals": [], "pcg_iters": []}
    u = np.zeros(disc.mesh.ndof) if u0 is None else u0.copy()
    u, ok = _newton(disc, u, lambda v: Pext - disc.internal_force(v), 0.0, tol, pcg_rtol,
                    maxnewton, linear, np.linalg.norm(Pext), stats)
    stats["converged"] = ok
    return u, stats


def initial_acceleration(disc, u0, P0):
    """a_0 = M^{-1} (P_0 - R(u_0)) with constrained rows zeroed (Sec. 4.1)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    M = disc.mass_matrix()
    keep = sp.diags((~disc.mask).astype(float))
    Mm = keep @ M @ keep + sp.diags(disc.mask.astype(float))
    rhs = P0 - disc.internal_force(u0)
    rhs[disc.mask] = 0.0
    return spla.spsolve(Mm.tocsc(), rhs)


def _masked_mass(disc):
    """Consistent mass with constrained rows/columns replaced by identity."""
    import scipy.sparse as sp
    M = disc.mass_matrix()
    keep = sp.diags((~disc.mask).astype(float))
    return (keep @ M @ keep + sp.diags(disc.mask.astype(float))).tocsc()


def mass_solve(disc, rhs, linear="direct", rtol=1e-13, Mm=None):
    """a = M^{-1} rhs on free DOFs (constrained entries 0)."""
    rhs = np.where(disc.mask, 0.0, rhs)
    if linear == "direct":
        import scipy.sparse.linalg as spla
        return spla.spsolve(Mm if Mm is not None else _masked_mass(disc), rhs)
    d = np.where(disc.mask, 1.0, disc.mass_diagonal())
    a, _, _ = jacobi_pcg(lambda x: np.where(disc.mask, x, disc.mass_apply(np.where(disc.mask, 0.0, x))), rhs, d,
                         rtol)
    return a


def central_difference_start(disc, u0, v0, P0, dt, linear="direct"):
    """Start-up of the central-difference scheme (Sec. 4.1):
    a_0 = M^{-1} (P_0 - R(u_0)),  u_{-1} = u_0 - dt v_0 + dt^2 / 2 a_0."""
    a0 = mass_solve(disc, P0 - disc.internal_force(u0), linear)
    return u0 - dt * v0 + 0.5 * dt * dt * a0, a0


def central_difference_step(disc, u, u_prev, Pn, dt, linear="direct", Mm=None):
    """One explicit step (Sec. 4.1, eq. Motion_explicit2):
    (M / dt^2) u_{n+1} = P_n - R(u_n) + (M / dt^2)(2 u_n - u_{n-1}),
    solved as M a_n = P_n - R(u_n), u_{n+1} = 2 u_n - u_{n-1} + dt^2 a_n.
    Constrained DOFs keep their values.  Returns (u_{n+1}, a_n)."""
    a = mass_solve(disc, Pn - disc.internal_force(u), linear, Mm=Mm)
    unew = 2.0 * u - u_prev + dt * dt * a
    unew[disc.mask] = u[disc.mask]
    return unew, a
