"""Thin Python binding over the libsdme C ABI (include/sdme.h).

Argument marshalling only: every step of the hot path runs in the library's
sm_103a kernels.  Vectors are passed as torch CUDA float64 tensors (their
device pointers); the library never sees torch types.  Importing this
package loads libsdme.so and fails loudly when it is missing or was built
without the entry points the header declares.

Method: Dias, Suzuki, Valente, Bittencourt (arXiv:2104.13466): SDME 1D bases
(Sec. 2), total-Lagrangian neo-Hookean elastodynamics (Sec. 3), Newmark +
Newton with diagonal-preconditioned CG (Sec. 4.2, Sec. 5).
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsdme.so")

# status codes (sdme_status)
OK, EINVAL, ENOMEM, ECUDA, PCG_MAXIT, NEWTON_DIVERGED, NONPOSITIVE_J, NAN, TIMEOUT, EUNSUPPORTED = range(10)
# basis kinds (sdme_basis_kind)
NODAL, MODAL, SDME_M, SDME_K, SDME_H, NODAL_LUMPED = range(6)
KIND_NAMES = {"nodal": NODAL, "modal": MODAL, "sdme_m": SDME_M, "sdme_k": SDME_K, "sdme_h": SDME_H,
              "nodal_lumped": NODAL_LUMPED}
# precisions (sdme_precision)
FP64, MIXED_FP32 = 0, 1
# faces
XMIN, XMAX, YMIN, YMAX, ZMIN, ZMAX = range(6)
FACE_NAMES = {"xmin": XMIN, "xmax": XMAX, "ymin": YMIN, "ymax": YMAX, "zmin": ZMIN, "zmax": ZMAX}

EXPORTS = ("sdme_status_string", "sdme_build_basis1d", "sdme_create", "sdme_destroy", "sdme_get_sizes",
           "sdme_internal_force", "sdme_mass_apply", "sdme_tangent_apply", "sdme_diagonal", "sdme_pcg_solve",
           "sdme_traction_load", "sdme_implicit_newmark_step", "sdme_set_timing", "sdme_get_timing",
           "sdme_tangent_apply_noalloc", "sdme_cuda_error_string", "sdme_explicit_start", "sdme_explicit_step",
           "sdme_energy", "sdme_estimate_dt_crit", "sdme_body_load", "sdme_mass_solve", "sdme_gauss_points",
           "sdme_set_material", "sdme_internal_force_vjp", "sdme_tape_create", "sdme_tape_destroy",
           "sdme_explicit_forward", "sdme_explicit_adjoint", "sdme_batch_create", "sdme_batch_destroy",
           "sdme_batch_layout", "sdme_batch_internal_force", "sdme_batch_tangent_apply", "sdme_batch_traction_load",
           "sdme_batch_newmark_step", "sdme_batch_tune", "sdme_batch_launches", "sdme_static_solve",
           "sdme_set_condensation", "sdme_set_refinement", "sdme_gauss_point_coords", "sdme_batch_set_persistent",
           "sdme_batch_persistent_info", "sdme_set_tangent_grid", "sdme_get_tangent_grid")


class BasisDesc(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int), ("kind", ctypes.c_int), ("k", ctypes.c_double), ("lam", ctypes.c_double),
                ("start_nodal", ctypes.c_int), ("jacobi_alpha", ctypes.c_double), ("jacobi_beta", ctypes.c_double)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("nelem", ctypes.c_int * 3), ("length", ctypes.c_double * 3), ("clamp", ctypes.c_uint * 6)]


class Material(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("lam", ctypes.c_double), ("rho", ctypes.c_double)]


class Problem(ctypes.Structure):
    _fields_ = [("mesh", MeshDesc), ("mat", Material), ("P", ctypes.c_int)]


class NewtonOpts(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("gamma", ctypes.c_double), ("newton_tol", ctypes.c_double),
                ("max_newton", ctypes.c_int), ("pcg_rtol", ctypes.c_double), ("mixed_rtol", ctypes.c_double),
                ("pcg_maxit", ctypes.c_int), ("forcing", ctypes.c_int)]


class StepStats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("pcg_iters_total", ctypes.c_int), ("matvecs", ctypes.c_int),
                ("converged", ctypes.c_int), ("residual0", ctypes.c_double), ("residual_final", ctypes.c_double),
                ("pcg_iters", ctypes.c_int * 32), ("residuals", ctypes.c_double * 33),
                ("residual_ref", ctypes.c_double), ("refine_sweeps", ctypes.c_int), ("lin_rel_max", ctypes.c_double)]


class State(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("a", ctypes.c_void_p)]


class ExplicitState(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("u_prev", ctypes.c_void_p), ("a", ctypes.c_void_p)]


class Timing(ctypes.Structure):
    _fields_ = [("tangent_ms", ctypes.c_double), ("tangent_launches", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsdme.so not built at %s; run `python paper_2104_13466_gb300/build.py` "
                          "(there is no CPU fallback)" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name in EXPORTS:
        if not hasattr(lib, name):
            raise ImportError("libsdme.so lacks %s" % name)
    vp, d, i, pd = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    lib.sdme_status_string.restype = ctypes.c_char_p
    lib.sdme_status_string.argtypes = [i]
    lib.sdme_cuda_error_string.restype = ctypes.c_char_p
    lib.sdme_cuda_error_string.argtypes = [vp]
    lib.sdme_build_basis1d.argtypes = [ctypes.POINTER(BasisDesc), i, pd, pd, pd, pd, pd, pd]
    lib.sdme_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(MeshDesc), ctypes.POINTER(Material),
                                ctypes.POINTER(BasisDesc), i, vp]
    lib.sdme_destroy.argtypes = [vp]
    lib.sdme_get_sizes.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int64)]
    lib.sdme_internal_force.argtypes = [vp, vp, vp]
    lib.sdme_mass_apply.argtypes = [vp, vp, vp]
    lib.sdme_tangent_apply.argtypes = [vp, vp, d, vp, vp]
    lib.sdme_diagonal.argtypes = [vp, vp, d, vp]
    lib.sdme_pcg_solve.argtypes = [vp, vp, d, vp, vp, d, i, ctypes.POINTER(i), pd]
    lib.sdme_traction_load.argtypes = [vp, i, pd, vp]
    lib.sdme_implicit_newmark_step.argtypes = [vp, ctypes.POINTER(State), d, vp, ctypes.POINTER(NewtonOpts),
                                               ctypes.POINTER(StepStats)]
    lib.sdme_explicit_start.argtypes = [vp, ctypes.POINTER(ExplicitState), d, vp, vp, d, i]
    lib.sdme_explicit_step.argtypes = [vp, ctypes.POINTER(ExplicitState), d, vp, d, i, ctypes.POINTER(i)]
    lib.sdme_energy.argtypes = [vp, vp, vp, pd, pd]
    lib.sdme_estimate_dt_crit.argtypes = [vp, vp, i, pd, pd]
    lib.sdme_body_load.argtypes = [vp, vp, vp]
    lib.sdme_mass_solve.argtypes = [vp, vp, vp, d, i, ctypes.POINTER(i), pd]
    lib.sdme_gauss_points.argtypes = [vp, pd, pd]
    lib.sdme_set_material.argtypes = [vp, ctypes.POINTER(Material)]
    lib.sdme_internal_force_vjp.argtypes = [vp, vp, vp, vp, pd, pd]
    lib.sdme_tape_create.argtypes = [vp, i, i, ctypes.POINTER(vp)]
    lib.sdme_tape_destroy.argtypes = [vp]
    lib.sdme_explicit_forward.argtypes = [vp, vp, d, vp, vp, vp, pd, d, i, vp]
    lib.sdme_explicit_adjoint.argtypes = [vp, vp, vp, pd, pd, vp, vp, vp]
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.sdme_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Problem), i, ctypes.POINTER(BasisDesc), i, vp]
    lib.sdme_batch_destroy.argtypes = [vp]
    lib.sdme_batch_layout.argtypes = [vp, i64p, i64p, i64p]
    lib.sdme_batch_internal_force.argtypes = [vp, vp, vp]
    lib.sdme_batch_tangent_apply.argtypes = [vp, vp, d, vp, vp]
    lib.sdme_batch_traction_load.argtypes = [vp, i, pd, vp]
    lib.sdme_batch_newmark_step.argtypes = [vp, ctypes.POINTER(State), d, vp, ctypes.POINTER(NewtonOpts),
                                            ctypes.POINTER(StepStats)]
    lib.sdme_batch_tune.argtypes = [vp, i, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                    ctypes.POINTER(ctypes.c_float)]
    lib.sdme_batch_launches.argtypes = [vp, i64p]
    lib.sdme_static_solve.argtypes = [vp, vp, vp, ctypes.POINTER(NewtonOpts), ctypes.POINTER(StepStats)]
    lib.sdme_set_condensation.argtypes = [vp, i]
    lib.sdme_set_timing.argtypes = [vp, i]
    lib.sdme_set_refinement.argtypes = [vp, i]
    lib.sdme_gauss_point_coords.argtypes = [vp, vp]
    lib.sdme_batch_set_persistent.argtypes = [vp, i, ctypes.POINTER(i)]
    lib.sdme_set_tangent_grid.argtypes = [vp, i]
    lib.sdme_get_tangent_grid.argtypes = [vp]
    lib.sdme_batch_persistent_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_float),
                                               ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    lib.sdme_get_timing.argtypes = [vp, ctypes.POINTER(Timing)]
    lib.sdme_tangent_apply_noalloc.argtypes = [ctypes.POINTER(MeshDesc), ctypes.POINTER(Material), i, pd, pd, pd,
                                               pd, vp, d, vp, vp, vp]
    for name in EXPORTS:
        if name not in ("sdme_status_string", "sdme_cuda_error_string"):
            getattr(lib, name).restype = ctypes.c_int
    return lib


lib = _load()


class SdmeError(RuntimeError):
    def __init__(self, status, where, detail=None):
        self.status = status
        msg = "%s: %s (%d)" % (where, lib.sdme_status_string(status).decode(), status)
        if detail:
            msg += ": " + detail
        super().__init__(msg)


def _check(status, where, allow=(), ctx=None):
    if status != OK and status not in allow:
        detail = None
        if status == ECUDA and ctx is not None:
            detail = lib.sdme_cuda_error_string(ctx).decode()
        raise SdmeError(status, where, detail)
    return status


def _ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    if not t.is_cuda or t.dtype.itemsize != 8 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def basis_desc(P, kind, k=0.5, lam=100.0, start_nodal=False, jacobi_alpha=1.0, jacobi_beta=1.0):
    kind = KIND_NAMES[kind] if isinstance(kind, str) else int(kind)
    return BasisDesc(int(P), kind, float(k), float(lam), int(bool(start_nodal)), float(jacobi_alpha),
                     float(jacobi_beta))


def build_basis1d(P, kind, Q=None, k=0.5, lam=100.0, start_nodal=False):
    """Host-only 1D basis tables (lattice order); returns numpy arrays
    (xq, wq, B, D, M1, K1)."""
    import numpy as np
    Q = Q or (P + 2)
    n = P + 1
    out = [np.zeros(Q), np.zeros(Q), np.zeros(Q * n), np.zeros(Q * n), np.zeros(n * n), np.zeros(n * n)]
    ptrs = [o.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for o in out]
    desc = basis_desc(P, kind, k, lam, start_nodal)
    _check(lib.sdme_build_basis1d(ctypes.byref(desc), int(Q), *ptrs), "sdme_build_basis1d")
    xq, wq, B, D, M1, K1 = out
    return xq, wq, B.reshape(Q, n), D.reshape(Q, n), M1.reshape(n, n), K1.reshape(n, n)


def mesh_desc(elems, lengths, clamp):
    """clamp: dict face-name -> iterable of components.  Two-entry elems and
    lengths describe a plane-strain rectangle of quadrilaterals (nelem[2] = 0)."""
    m = MeshDesc()
    for d in range(3):
        m.nelem[d] = int(elems[d]) if d < len(elems) else 0
        m.length[d] = float(lengths[d]) if d < len(lengths) else 1.0
    for f, comps in (clamp or {}).items():
        bits = 0
        for c in comps:
            bits |= 1 << int(c)
        m.clamp[FACE_NAMES[f] if isinstance(f, str) else int(f)] = bits
    return m


def tangent_apply_noalloc(elems, lengths, clamp, mu, lam, rho, P, tables, u, b1, x, y, stream=None):
    """sdme_tangent_apply_noalloc: float64 tangent matvec without a context
    and without any allocation; ``tables`` = (xq, wq, B, D) as returned by
    build_basis1d (float64 numpy arrays)."""
    import numpy as np
    import torch
    mesh = mesh_desc(elems, lengths, clamp)
    mat = Material(float(mu), float(lam), float(rho))
    arrs = [np.ascontiguousarray(t, dtype=np.float64) for t in tables]
    ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrs]
    stream = stream or torch.cuda.current_stream()
    return _check(lib.sdme_tangent_apply_noalloc(ctypes.byref(mesh), ctypes.byref(mat), int(P), *ptrs, _ptr(u),
                                                 float(b1), _ptr(x), _ptr(y), ctypes.c_void_p(stream.cuda_stream)),
                  "sdme_tangent_apply_noalloc", "sdme_cuda_error_string", "sdme_explicit_start", "sdme_explicit_step",
           "sdme_energy", "sdme_estimate_dt_crit", "sdme_body_load", "sdme_mass_solve", "sdme_gauss_points")


def _stats_dict(stats, status):
    n = min(stats.newton_iters, 32)
    ref = stats.residual_ref
    return {"status": status, "newton_iters": stats.newton_iters, "pcg_iters_total": stats.pcg_iters_total,
            "matvecs": stats.matvecs, "converged": bool(stats.converged), "residual0": stats.residual0,
            "residual_final": stats.residual_final, "residual_ref": ref,
            "residual_rel": stats.residual_final / ref if ref > 0 else 0.0,
            "refine_sweeps": stats.refine_sweeps, "lin_rel_max": stats.lin_rel_max,
            "pcg_iters": list(stats.pcg_iters[:n]), "residuals": list(stats.residuals[:n + 1])}


class _ExplicitStateHolder:
    """Keeps the tensors of an sdme_explicit_state alive and tracks which
    tensor currently holds u_n and u_{n-1} after the library swaps them."""

    def __init__(self, u, u_prev, a):
        self._t = {u.data_ptr(): u, u_prev.data_ptr(): u_prev}
        self.a = a
        self.c = ExplicitState(u.data_ptr(), u_prev.data_ptr(), a.data_ptr())
        self.sync()

    def sync(self):
        self.u = self._t[self.c.u]
        self.u_prev = self._t[self.c.u_prev]


class Context:
    """Owns an sdme_ctx.  Methods mirror the C entry points."""

    def __init__(self, elems, lengths, clamp, mu, lam, rho, P, kind, precision=FP64, k=0.5, lam_h=100.0,
                 start_nodal=False, stream=None):
        import torch
        self._mesh = mesh_desc(elems, lengths, clamp)
        self._mat = Material(float(mu), float(lam), float(rho))
        self._basis = basis_desc(P, kind, k, lam_h, start_nodal)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib.sdme_create(ctypes.byref(h), ctypes.byref(self._mesh), ctypes.byref(self._mat),
                               ctypes.byref(self._basis), int(precision), ctypes.c_void_p(stream.cuda_stream)),
               "sdme_create")
        self._h = h
        ndof = ctypes.c_int64()
        N = (ctypes.c_int * 3)()
        ne = ctypes.c_int64()
        _check(lib.sdme_get_sizes(h, ctypes.byref(ndof), N, ctypes.byref(ne)), "sdme_get_sizes")
        self.ndof, self.N, self.nelem = ndof.value, tuple(N), ne.value
        self.P = P

    def close(self):
        if getattr(self, "_h", None):
            lib.sdme_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def internal_force(self, u, R):
        return _check(lib.sdme_internal_force(self._h, _ptr(u), _ptr(R)), "sdme_internal_force", ctx=self._h)

    def set_material(self, mu, lam, rho=None):
        m = Material(float(mu), float(lam), float(self._mat.rho if rho is None else rho))
        _check(lib.sdme_set_material(self._h, ctypes.byref(m)), "sdme_set_material")
        self._mat = m

    @property
    def material(self):
        return self._mat.mu, self._mat.lam, self._mat.rho

    def internal_force_vjp(self, u, w, gu):
        """gu = (dR/du)^T w (overwritten); returns (w . dR/dmu, w . dR/dlambda)."""
        gmu, glam = ctypes.c_double(), ctypes.c_double()
        _check(lib.sdme_internal_force_vjp(self._h, _ptr(u), _ptr(w), _ptr(gu), ctypes.byref(gmu),
                                           ctypes.byref(glam)), "sdme_internal_force_vjp", ctx=self._h)
        return gmu.value, glam.value

    def mass_apply(self, x, y):
        return _check(lib.sdme_mass_apply(self._h, _ptr(x), _ptr(y)), "sdme_mass_apply", ctx=self._h)

    def tangent_apply(self, u, b1, x, y):
        return _check(lib.sdme_tangent_apply(self._h, _ptr(u), float(b1), _ptr(x), _ptr(y)), "sdme_tangent_apply", ctx=self._h)

    def diagonal(self, u, b1, d):
        return _check(lib.sdme_diagonal(self._h, _ptr(u), float(b1), _ptr(d)), "sdme_diagonal", ctx=self._h)

    def pcg_solve(self, u, b1, b, x, rtol=1e-10, maxit=20000, allow_maxit=False):
        its = ctypes.c_int()
        rel = ctypes.c_double()
        st = lib.sdme_pcg_solve(self._h, _ptr(u), float(b1), _ptr(b), _ptr(x), float(rtol), int(maxit),
                                ctypes.byref(its), ctypes.byref(rel))
        _check(st, "sdme_pcg_solve", allow=(PCG_MAXIT,) if allow_maxit else (), ctx=self._h)
        return its.value, rel.value

    def traction_load(self, face, t, f):
        face = FACE_NAMES[face] if isinstance(face, str) else int(face)
        tt = (ctypes.c_double * 3)(*[float(v) for v in t])
        return _check(lib.sdme_traction_load(self._h, face, tt, _ptr(f)), "sdme_traction_load", ctx=self._h)

    def implicit_newmark_step(self, u, v, a, dt, P_next, beta=0.25, gamma=0.5, newton_tol=1e-8, max_newton=30,
                              pcg_rtol=1e-10, mixed_rtol=1e-4, pcg_maxit=20000, forcing=0, allow=()):
        st = State(u.data_ptr(), v.data_ptr(), a.data_ptr())
        for t in (u, v, a):
            _ptr(t)
        opts = NewtonOpts(beta, gamma, newton_tol, max_newton, pcg_rtol, mixed_rtol, pcg_maxit, int(forcing))
        stats = StepStats()
        status = lib.sdme_implicit_newmark_step(self._h, ctypes.byref(st), float(dt), _ptr(P_next),
                                                ctypes.byref(opts), ctypes.byref(stats))
        _check(status, "sdme_implicit_newmark_step", allow=allow, ctx=self._h)
        return _stats_dict(stats, status)

    def set_condensation(self, enable=True):
        """Static condensation of the element-interior modes for every
        effective-operator solve (sdme_set_condensation)."""
        return _check(lib.sdme_set_condensation(self._h, int(bool(enable))), "sdme_set_condensation", ctx=self._h)

    def static_solve(self, u, P, newton_tol=1e-8, max_newton=50, pcg_rtol=1e-12, mixed_rtol=1e-4, pcg_maxit=20000,
                     forcing=0, allow=()):
        """R(u) = P by Newton-Raphson (u: initial guess in, solution out)."""
        opts = NewtonOpts(0.25, 0.5, newton_tol, max_newton, pcg_rtol, mixed_rtol, pcg_maxit, int(forcing))
        stats = StepStats()
        status = lib.sdme_static_solve(self._h, _ptr(u), _ptr(P), ctypes.byref(opts), ctypes.byref(stats))
        _check(status, "sdme_static_solve", allow=allow, ctx=self._h)
        return _stats_dict(stats, status)

    # -- explicit central difference (Sec. 4.1) ------------------------------
    def explicit_state(self, u, u_prev, a):
        """Bundle three float64 CUDA tensors (u_n, u_{n-1}, a_n) for the
        explicit calls; the calls swap which tensor holds u and u_prev, read
        the current assignment from ``current()``."""
        for t in (u, u_prev, a):
            _ptr(t)
        return _ExplicitStateHolder(u, u_prev, a)

    def explicit_start(self, st, dt, P0, v0, rtol=1e-12, maxit=20000):
        return _check(lib.sdme_explicit_start(self._h, ctypes.byref(st.c), float(dt), _ptr(P0), _ptr(v0),
                                              float(rtol), int(maxit)), "sdme_explicit_start", ctx=self._h)

    def explicit_step(self, st, dt, Pn, rtol=1e-12, maxit=20000):
        its = ctypes.c_int()
        _check(lib.sdme_explicit_step(self._h, ctypes.byref(st.c), float(dt), _ptr(Pn), float(rtol), int(maxit),
                                      ctypes.byref(its)), "sdme_explicit_step", ctx=self._h)
        st.sync()
        return its.value

    def energy(self, u=None, v=None):
        ke = ctypes.c_double()
        se = ctypes.c_double()
        _check(lib.sdme_energy(self._h, _ptr(u) if u is not None else None, _ptr(v) if v is not None else None,
                               ctypes.byref(ke) if v is not None else None,
                               ctypes.byref(se) if u is not None else None), "sdme_energy", ctx=self._h)
        return (ke.value if v is not None else None), (se.value if u is not None else None)

    def estimate_dt_crit(self, u, iters=50):
        dt = ctypes.c_double()
        lam = ctypes.c_double()
        _check(lib.sdme_estimate_dt_crit(self._h, _ptr(u), int(iters), ctypes.byref(dt), ctypes.byref(lam)),
               "sdme_estimate_dt_crit", ctx=self._h)
        return dt.value, lam.value

    def gauss_points(self):
        import numpy as np
        Q = self.P + 2
        xq, wq = np.zeros(Q), np.zeros(Q)
        _check(lib.sdme_gauss_points(self._h, xq.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     wq.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "sdme_gauss_points")
        return xq, wq

    def gauss_point_coords(self, elems=None, lengths=None):
        """Physical coordinates (torch CUDA float64, [nelem][Q^3][3]) of the
        Gauss points in the layout sdme_body_load expects
        (sdme_gauss_point_coords; the mesh is the context's own, the
        arguments are accepted for compatibility and ignored)."""
        import torch
        Q = self.P + 2
        X = torch.empty((self.nelem, Q ** 3, 3), dtype=torch.float64, device="cuda")
        _check(lib.sdme_gauss_point_coords(self._h, _ptr(X)), "sdme_gauss_point_coords", ctx=self._h)
        return X

    def body_load(self, fq, f):
        return _check(lib.sdme_body_load(self._h, _ptr(fq), _ptr(f)), "sdme_body_load", ctx=self._h)

    def mass_solve(self, b, x, rtol=1e-12, maxit=20000):
        its = ctypes.c_int()
        rel = ctypes.c_double()
        _check(lib.sdme_mass_solve(self._h, _ptr(b), _ptr(x), float(rtol), int(maxit), ctypes.byref(its),
                                   ctypes.byref(rel)), "sdme_mass_solve", ctx=self._h)
        return its.value, rel.value

    def set_timing(self, enable=True):
        return _check(lib.sdme_set_timing(self._h, int(bool(enable))), "sdme_set_timing")

    def set_tangent_grid(self, ctas):
        """CTAs of the PCG tangent launch: 0 one per element, -1 the resident
        CTAs, > 0 that many (sdme_set_tangent_grid); returns the grid in use."""
        _check(lib.sdme_set_tangent_grid(self._h, int(ctas)), "sdme_set_tangent_grid", ctx=self._h)
        return lib.sdme_get_tangent_grid(self._h)

    def set_refinement(self, max_restarts):
        """Float64-residual restarts allowed per float32 PCG solve (0: off)."""
        return _check(lib.sdme_set_refinement(self._h, int(max_restarts)), "sdme_set_refinement")

    def timing(self):
        t = Timing()
        _check(lib.sdme_get_timing(self._h, ctypes.byref(t)), "sdme_get_timing")
        return {"tangent_ms": t.tangent_ms, "tangent_launches": t.tangent_launches,
                "kernel_launches": t.kernel_launches}


def _material_grad(x, g):
    """Gradient g (a float) in the type of the material input x."""
    import torch
    if isinstance(x, torch.Tensor) and x.requires_grad:
        return torch.tensor(g, dtype=x.dtype, device=x.device).reshape(x.shape)
    return None


def _InternalForceFunction():
    import torch

    class InternalForce(torch.autograd.Function):
        """R(u; mu, lambda) of sdme_internal_force with the hand-written
        adjoint of sdme_internal_force_vjp as its backward."""

        @staticmethod
        def forward(fctx, ctx, u, mu, lam):
            ctx.set_material(float(mu), float(lam))
            R = torch.empty_like(u)
            ctx.internal_force(u, R)
            fctx.sdme = ctx
            fctx.mat = (float(mu), float(lam))
            fctx.mu_in, fctx.lam_in = mu, lam
            fctx.save_for_backward(u)
            return R

        @staticmethod
        def backward(fctx, gR):
            (u,) = fctx.saved_tensors
            ctx = fctx.sdme
            ctx.set_material(*fctx.mat)
            gu = torch.empty_like(u)
            gmu, glam = ctx.internal_force_vjp(u, gR.contiguous(), gu)
            return None, gu, _material_grad(fctx.mu_in, gmu), _material_grad(fctx.lam_in, glam)

    return InternalForce


_internal_force_fn = None


def internal_force(ctx, u, mu, lam):
    """Differentiable internal force R(u; mu, lambda) (float64 CUDA u; mu and
    lam floats or 0-dim tensors).  Sets the context's material to (mu, lam)."""
    global _internal_force_fn
    if _internal_force_fn is None:
        _internal_force_fn = _InternalForceFunction()
    return _internal_force_fn.apply(ctx, u, mu, lam)


class Tape:
    """Owns an sdme_tape: a checkpointed explicit trajectory of ``ctx``
    (``nsteps`` steps, checkpoints every ``every`` steps) and its adjoint."""

    def __init__(self, ctx, nsteps, every):
        h = ctypes.c_void_p()
        _check(lib.sdme_tape_create(ctx._h, int(nsteps), int(every), ctypes.byref(h)), "sdme_tape_create",
               ctx=ctx._h)
        self._h, self.ctx, self.nsteps, self.every = h, ctx, int(nsteps), int(every)

    def close(self):
        if getattr(self, "_h", None):
            lib.sdme_tape_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, dt, u0, v0, uN, f=None, s=None, rtol=1e-12, maxit=20000):
        """Runs the trajectory; writes u_N into uN.  Loads P_n = s[n] f."""
        import numpy as np
        sp = None
        if f is not None:
            s = np.ascontiguousarray(np.broadcast_to(np.asarray(1.0 if s is None else s, dtype=np.float64),
                                                     (self.nsteps,)))
            self._s = s
            sp = s.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib.sdme_explicit_forward(self.ctx._h, self._h, float(dt), _ptr(u0), _ptr(v0),
                                         _ptr(f) if f is not None else None, sp, float(rtol), int(maxit),
                                         _ptr(uN)), "sdme_explicit_forward", ctx=self.ctx._h)

    def adjoint(self, gN, gu0=None, gv0=None, gf=None):
        """Reverse sweep for dJ/du_N = gN; fills the given device vectors and
        returns (dJ/dmu, dJ/dlambda)."""
        gmu, glam = ctypes.c_double(), ctypes.c_double()
        opt = [_ptr(t) if t is not None else None for t in (gu0, gv0, gf)]
        _check(lib.sdme_explicit_adjoint(self.ctx._h, self._h, _ptr(gN), ctypes.byref(gmu), ctypes.byref(glam),
                                         *opt), "sdme_explicit_adjoint", ctx=self.ctx._h)
        return gmu.value, glam.value


def _TrajectoryFunction():
    import torch

    class ExplicitTrajectory(torch.autograd.Function):
        """u_N of a checkpointed explicit trajectory as a function of
        (u0, v0, f, mu, lambda); backward is the hand-written discrete adjoint."""

        @staticmethod
        def forward(fctx, tape, dt, s, rtol, u0, v0, f, mu, lam):
            ctx = tape.ctx
            ctx.set_material(float(mu), float(lam))
            uN = torch.empty_like(u0)
            tape.forward(dt, u0, v0, uN, f=f, s=s, rtol=rtol)
            fctx.tape, fctx.mat = tape, (float(mu), float(lam))
            fctx.mu_in, fctx.lam_in, fctx.has_f = mu, lam, f is not None
            return uN

        @staticmethod
        def backward(fctx, gN):
            tape = fctx.tape
            tape.ctx.set_material(*fctx.mat)
            need = fctx.needs_input_grad
            gu0 = torch.empty_like(gN) if need[4] else None
            gv0 = torch.empty_like(gN) if need[5] else None
            gf = torch.empty_like(gN) if (need[6] and fctx.has_f) else None
            gmu, glam = tape.adjoint(gN.contiguous(), gu0, gv0, gf)
            return (None, None, None, None, gu0, gv0, gf, _material_grad(fctx.mu_in, gmu),
                    _material_grad(fctx.lam_in, glam))

    return ExplicitTrajectory


_trajectory_fn = None


def explicit_trajectory(tape, dt, u0, v0, mu, lam, f=None, s=None, rtol=1e-12):
    """Differentiable u_N of the explicit scheme (start-up from (u0, v0),
    tape.nsteps steps, loads s[n] f).  Backward runs the discrete adjoint on
    the tape; the tape holds one trajectory, so call backward before the
    next forward on the same tape."""
    global _trajectory_fn
    if _trajectory_fn is None:
        _trajectory_fn = _TrajectoryFunction()
    return _trajectory_fn.apply(tape, dt, s, rtol, u0, v0, f, mu, lam)


class Batch:
    """Owns an sdme_batch: independent box-mesh problems solved together.
    ``problems``: iterable of dicts with keys elems, lengths, clamp, mu, lam,
    rho, P.  Vectors are concatenated float64 CUDA tensors of ``total`` entries;
    problem i occupies [offsets[i], offsets[i] + ndofs[i])."""

    def __init__(self, problems, kind, precision=FP64, k=0.5, lam_h=100.0, start_nodal=False, stream=None):
        import torch
        problems = list(problems)
        arr = (Problem * len(problems))()
        for j, pr in enumerate(problems):
            arr[j].mesh = mesh_desc(pr["elems"], pr["lengths"], pr["clamp"])
            arr[j].mat = Material(float(pr["mu"]), float(pr["lam"]), float(pr.get("rho", 1.0)))
            arr[j].P = int(pr["P"])
        self._basis = basis_desc(1, kind, k, lam_h, start_nodal)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib.sdme_batch_create(ctypes.byref(h), arr, len(problems), ctypes.byref(self._basis), int(precision),
                                     ctypes.c_void_p(stream.cuda_stream)), "sdme_batch_create")
        self._h = h
        self.nprob = len(problems)
        tot = ctypes.c_int64()
        off = (ctypes.c_int64 * self.nprob)()
        nd = (ctypes.c_int64 * self.nprob)()
        _check(lib.sdme_batch_layout(h, ctypes.byref(tot), off, nd), "sdme_batch_layout")
        self.total, self.offsets, self.ndofs = tot.value, list(off), list(nd)

    def close(self):
        if getattr(self, "_h", None):
            lib.sdme_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def zeros(self):
        import torch
        return torch.zeros(self.total, dtype=torch.float64, device="cuda")

    def segment(self, v, i):
        return v[self.offsets[i]:self.offsets[i] + self.ndofs[i]]

    def internal_force(self, u, R):
        return _check(lib.sdme_batch_internal_force(self._h, _ptr(u), _ptr(R)), "sdme_batch_internal_force")

    def tangent_apply(self, u, b1, x, y):
        return _check(lib.sdme_batch_tangent_apply(self._h, _ptr(u), float(b1), _ptr(x), _ptr(y)),
                      "sdme_batch_tangent_apply")

    def traction_load(self, face, t, f):
        """t: sequence of nprob 3-vectors (or one 3-vector for all)."""
        import numpy as np
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(t, dtype=np.float64), (self.nprob, 3)))
        face = FACE_NAMES[face] if isinstance(face, str) else int(face)
        return _check(lib.sdme_batch_traction_load(self._h, face, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                   _ptr(f)), "sdme_batch_traction_load")

    def newmark_step(self, u, v, a, dt, P_next, beta=0.25, gamma=0.5, newton_tol=1e-8, max_newton=30,
                     pcg_rtol=1e-10, mixed_rtol=1e-4, pcg_maxit=20000, forcing=0, allow=()):
        st = State(u.data_ptr(), v.data_ptr(), a.data_ptr())
        for t in (u, v, a):
            _ptr(t)
        opts = NewtonOpts(beta, gamma, newton_tol, max_newton, pcg_rtol, mixed_rtol, pcg_maxit, int(forcing))
        stats = (StepStats * self.nprob)()
        status = lib.sdme_batch_newmark_step(self._h, ctypes.byref(st), float(dt), _ptr(P_next), ctypes.byref(opts),
                                             stats)
        _check(status, "sdme_batch_newmark_step", allow=allow)
        return [_stats_dict(s, status) for s in stats]

    def tune(self, reps=5):
        """Launch-configuration tuner; returns [(P, grid, ms per launch)] per order group."""
        m = 16
        ng = ctypes.c_int()
        orders, grids, ms = (ctypes.c_int * m)(), (ctypes.c_int * m)(), (ctypes.c_float * m)()
        _check(lib.sdme_batch_tune(self._h, int(reps), m, ctypes.byref(ng), orders, grids, ms), "sdme_batch_tune")
        return [(orders[j], grids[j], ms[j]) for j in range(min(ng.value, m))]

    def launches(self):
        n = ctypes.c_int64()
        _check(lib.sdme_batch_launches(self._h, ctypes.byref(n)), "sdme_batch_launches")
        return n.value

    def set_persistent(self, mode, kper=None):
        """PCG operator as one persistent launch across the order groups:
        mode 1 always, 0 never, -1 as the tuner decides; kper: {P: elements
        per work item} (orders not given keep 1)."""
        arr = None
        if kper is not None:
            arr = (ctypes.c_int * 9)(*[int(kper.get(P, 1)) if P else 0 for P in range(9)])
        return _check(lib.sdme_batch_set_persistent(self._h, int(mode), arr), "sdme_batch_set_persistent")

    def persistent_info(self):
        on = ctypes.c_int()
        kper = (ctypes.c_int * 9)()
        pm, gm = ctypes.c_float(), ctypes.c_float()
        om = (ctypes.c_float * 9)()
        _check(lib.sdme_batch_persistent_info(self._h, ctypes.byref(on), kper, ctypes.byref(pm), ctypes.byref(gm),
                                              om), "sdme_batch_persistent_info")
        return {"on": bool(on.value), "kper": {P: kper[P] for P in range(1, 9)}, "persist_ms": pm.value,
                "groups_ms": gm.value, "order_ms": {P: om[P] for P in range(1, 9) if om[P] >= 0}}
