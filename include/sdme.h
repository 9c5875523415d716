/*
 * sdme.h - C ABI of the GB300 matrix-free SDME / neo-Hookean Newton-PCG engine.
 *
 * Method: Dias, Suzuki, Valente, Bittencourt, "Simulation of non-linear
 * structural elastodynamic and impact problems using minimum energy and
 * simultaneous diagonalization high-order bases" (arXiv:2104.13466).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Mesh.  A box [0,Lx]x[0,Ly]x[0,Lz] split into nx x ny x nz equal hexahedra of
 *   order P (1 <= P <= 8), all with the same orientation.  The (P+1)^3
 *   coefficients of each element live on a global lattice of
 *   Nx x Ny x Nz = (nx P + 1) x (ny P + 1) x (nz P + 1) points; the 1D
 *   functions are ordered [vertex at -1, internal modes, vertex at +1].
 * Vectors.  Every global vector is float64, component-major
 *   ("structure of arrays"): index c*Nn + (iz*Ny + iy)*Nx + ix, c = 0,1,2,
 *   Nn = Nx*Ny*Nz, length ndof = 3*Nn.  Vector arguments named *_dev are
 *   device pointers (cudaMalloc'd or torch CUDA tensors) owned by the caller;
 *   they must not alias each other unless stated.
 * Streams.  All device work of a context is issued on the stream given to
 *   sdme_create.  Calls that return host scalars or check the device error
 *   word synchronise that stream; the others are stream-ordered.
 * Errors.  Every call returns an sdme_status; nothing throws or traps.  A
 *   sticky device error word (non-positive Jacobian) is checked at every
 *   host synchronisation and reported as SDME_NONPOSITIVE_J.
 * Dirichlet.  Homogeneous or prescribed values on whole box faces, per
 *   component (clamp[face] bit c).  A DOF is constrained when its lattice
 *   point lies on a clamped face: every 1D function except the vertex one
 *   vanishes there.
 */
#ifndef SDME_H
#define SDME_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SDME_OK = 0,
  SDME_EINVAL = 1,            /* bad argument */
  SDME_ENOMEM = 2,            /* device or host allocation failed */
  SDME_ECUDA = 3,             /* a CUDA runtime call failed */
  SDME_PCG_MAXIT = 4,         /* PCG reached maxit before rtol */
  SDME_NEWTON_DIVERGED = 5,   /* Newton reached max_newton before tol */
  SDME_NONPOSITIVE_J = 6,     /* det F <= 0 at some Gauss point */
  SDME_NAN = 7,               /* non-finite residual or PCG scalar */
  SDME_TIMEOUT = 8,           /* a bounded device-side wait gave up */
  SDME_EUNSUPPORTED = 9       /* order or option not built */
} sdme_status;

/* 1D expansion bases of Sec. 2. */
typedef enum {
  SDME_NODAL = 0,    /* Lagrange on GLL points, eqs. lagrangian / shape_functions_lag */
  SDME_MODAL = 1,    /* Jacobi modal ST basis, eq. BasePadrao1D */
  SDME_SDME_M = 2,   /* SD internal modes + ME vertex modes, L2 norm (eq. alphaMassa) */
  SDME_SDME_K = 3,   /* SD + ME, energy norm (eq. alphaRigidez) */
  SDME_SDME_H = 4,   /* SD + ME, Helmholtz norm K + lambda M (eq. alphaKN) */
  SDME_NODAL_LUMPED = 5 /* the nodal basis with its mass matrix integrated at its own
                           Gauss-Lobatto-Legendre nodes: diagonal (lumped) mass, the
                           diagonal-mass Lagrange variant of Sec. 5.2.1; stiffness and
                           loads as for SDME_NODAL.  Mass solves are divisions (no PCG);
                           operators with a mass term (b1 != 0) are SDME_EUNSUPPORTED. */
} sdme_basis_kind;

typedef enum {
  SDME_FP64 = 0,      /* everything in float64 */
  SDME_MIXED_FP32 = 1 /* tangent matvec, diagonal and PCG vectors in float32;
                         Newton residual, PCG scalars and time-integrator state
                         in float64.  PCG dot products: float32 products (of
                         float32 vectors, summed four at a time) accumulated
                         per thread in a compensated float32 (float-float,
                         about 48-bit) sum and reduced across threads in
                         float64; the operator's p.(A p) from float32
                         Gauss-point terms accumulated the same way.  The
                         refined tangent solves carry x as a float32
                         correction folded into a float64 solution at every
                         refinement check */
} sdme_precision;

enum { SDME_XMIN = 0, SDME_XMAX = 1, SDME_YMIN = 2, SDME_YMAX = 3, SDME_ZMIN = 4, SDME_ZMAX = 5 };

typedef struct {
  int P;                 /* polynomial order, 1..8 */
  sdme_basis_kind kind;
  double k;              /* SD parameter of eq. Y, in [0, 1] (paper: 0.5) */
  double lambda;         /* Helmholtz parameter of eq. EffectiveStiffness_lambda (paper: 100) */
  int start_nodal;       /* SDME kinds: build from the Lagrange (1) or Jacobi (0) basis */
  double jacobi_alpha;   /* modal weights of eq. BasePadrao1D (paper: 1, 1) */
  double jacobi_beta;
} sdme_basis_desc;

/*
 * Box meshes of equal hexahedra; nelem[2] = 0 selects a plane-strain
 * rectangle of equal quadrilaterals in the x-y plane instead (tensor products
 * of eq. ProdTensorialQuadrado; F_33 = 1): two components per lattice point,
 * vectors [2][Ny][Nx], clamp[4] = clamp[5] = 0, edges SDME_XMIN..SDME_YMAX.
 * Two-dimensional contexts support the internal force, tangent action,
 * diagonal, mass, PCG, static/Newmark/explicit steps, energy, critical step
 * and edge tractions; the adjoint, body loads, condensation, lumped mass and
 * batches are SDME_EUNSUPPORTED there.
 */
typedef struct {
  int nelem[3];          /* elements per direction (nelem[2] = 0: 2D) */
  double length[3];      /* box edge lengths (length[2] unused in 2D) */
  unsigned clamp[6];     /* per face (SDME_XMIN..SDME_ZMAX): bit c set = component c constrained */
} sdme_mesh_desc;

typedef struct {
  double mu, lambda;     /* Lame parameters of eq. hyperelastic strain energy */
  double rho;            /* reference density */
} sdme_material;

typedef struct {
  double beta, gamma;    /* Newmark parameters (reading of the garbled table: 0.25, 0.5) */
  double newton_tol;     /* stop when ||psi_k|| <= tol * max(||psi_0||, ||P||): the
                            paper's tolerance (Sec. 5.1) relative to the larger of
                            the step's initial residual and the applied load */
  int max_newton;
  double pcg_rtol;       /* FP64: ||r|| <= rtol ||b|| */
  double mixed_rtol;     /* MIXED_FP32: inner PCG tolerance (inexact Newton) */
  int pcg_maxit;
  int forcing;           /* 0: the inner tolerance above at every Newton iteration;
                            1: Eisenstat-Walker forcing terms (their "choice 2":
                            eta_k = 0.9 (|psi_k| / |psi_{k-1}|)^2 with the 0.9 eta^2
                            safeguard, eta_0 = eta_max = 0.01, no tighter than
                            0.5 tol |psi_0| / |psi_k|), never below the tolerance above.
                            The Newton test itself is unchanged. */
} sdme_newton_opts;

typedef struct {
  int newton_iters;
  int pcg_iters_total;
  int matvecs;                 /* tangent matvecs issued */
  int converged;               /* 1 if the Newton test was met */
  double residual0;            /* ||psi_0|| */
  double residual_final;       /* ||psi|| at exit */
  int pcg_iters[32];           /* per Newton iteration (first 32) */
  double residuals[33];        /* ||psi_k||, k = 0..min(newton_iters, 32) */
  double residual_ref;         /* max(||psi_0||, ||P||): the Newton test's reference */
  int refine_sweeps;           /* MIXED_FP32: float64 refinement restarts of the PCG solves */
  double lin_rel_max;          /* MIXED_FP32: largest float64 relative residual
                                  ||psi - (b1 M + K_T) du|| / ||psi|| of the step's solves */
} sdme_step_stats;

typedef struct {
  double* u;             /* displacement u_n (in) -> u_{n+1} (out), device */
  double* v;             /* velocity, device */
  double* a;             /* acceleration, device */
} sdme_state;

typedef struct sdme_ctx sdme_ctx;

/* Human-readable name of a status code (static storage). */
const char* sdme_status_string(sdme_status s);

/*
 * Host-only.  Build the 1D basis of Sec. 2 and tabulate it at Q Gauss-Legendre
 * points (Q >= 1; the device path uses Q = P + 2).  Steps: standard basis
 * (eq. shape_functions_lag or BasePadrao1D), 1D mass/stiffness (eqs.
 * Matrizesmassa, Matrizesrigidez), partition (eq. BlocosMassa), simultaneous
 * diagonalisation of the internal block (eqs. diagMassa, L, diagL, Y; each
 * internal function signed so that its derivative at -1 is positive and
 * ordered by ascending eigenvalue), minimum-energy vertex modes (eqs.
 * ExtensaoMEmassa, alphaMassa, alphaRigidez, alphaKN).
 * Outputs (caller-owned host arrays; any may be NULL), lattice order:
 *   xq[Q], wq[Q]          Gauss-Legendre points and weights on [-1, 1]
 *   B[Q*(P+1)]            B[q*(P+1)+j] = phi_j(xq[q])
 *   D[Q*(P+1)]            D[q*(P+1)+j] = phi_j'(xq[q])
 *   M1[(P+1)^2], K1[...]  1D mass and stiffness of the final basis
 * Returns SDME_EINVAL for P outside 1..8, Q outside 1..16 or a bad kind.
 */
sdme_status sdme_build_basis1d(const sdme_basis_desc* basis, int Q, double* xq, double* wq,
                               double* B, double* D, double* M1, double* K1);

/*
 * Create a context: builds the basis, uploads its tables, allocates device
 * work buffers (per-Gauss-point linearisation state, PCG vectors).  stream:
 * the cudaStream_t all of the context's work is issued on; NULL selects the
 * legacy default stream.  The stream is not owned and must outlive the
 * context.  Returns SDME_EINVAL for bad sizes/material/basis, SDME_ENOMEM
 * when a buffer cannot be allocated (nothing is leaked).
 */
sdme_status sdme_create(sdme_ctx** out, const sdme_mesh_desc* mesh, const sdme_material* mat,
                        const sdme_basis_desc* basis, sdme_precision prec, void* stream);

sdme_status sdme_destroy(sdme_ctx* ctx);

/* Sizes: ndof = 3*Nn, lattice dims N[3], element count. */
sdme_status sdme_get_sizes(const sdme_ctx* ctx, int64_t* ndof, int N[3], int64_t* nelem);

/*
 * R_dev = R(u), the internal force vector of eq. material virtual work
 * (second term, S : dE = P : grad du with P = F S of eq. second
 * Piolla_Kirchhoff relation), for every DOF (no Dirichlet treatment).
 * Also stores the linearisation state at u.  Always float64.
 */
sdme_status sdme_internal_force(sdme_ctx* ctx, const double* u_dev, double* R_dev);

/*
 * Replaces the material constants (mu, lambda, rho) of the context; sizes,
 * basis and buffers are kept.  Constraints as in sdme_create (mu > 0,
 * lambda >= 0, rho >= 0), else SDME_EINVAL and the context is unchanged.
 * Host-only, does not synchronise.
 */
sdme_status sdme_set_material(sdme_ctx* ctx, const sdme_material* mat);

/*
 * Vector-Jacobian product of the internal force R(u; mu, lambda) of
 * sdme_internal_force (Sec. 3: P = mu (F - F^{-T}) + lambda ln J F^{-T}):
 *   gu_dev   = (dR/du)^T w = K_T(u) w   (all DOFs, no Dirichlet treatment;
 *              K_T is the symmetric consistent tangent of Sec. 3.1),
 *   *gmu     = w . dR/dmu,   *glambda = w . dR/dlambda   (R is linear in both).
 * u_dev, w_dev, gu_dev: float64 device vectors of ndof entries, caller-owned;
 * gu_dev is overwritten.  gmu / glambda: host scalars, either may be NULL.
 * Always float64 (also in a MIXED_FP32 context).  Stores the linearisation
 * state at u.  Synchronises.  SDME_NONPOSITIVE_J if det F <= 0 at a Gauss point.
 */
sdme_status sdme_internal_force_vjp(sdme_ctx* ctx, const double* u_dev, const double* w_dev, double* gu_dev,
                                    double* gmu, double* glambda);

/* y_dev = M x_dev, consistent mass of eq. material virtual work (first term), no Dirichlet treatment. */
sdme_status sdme_mass_apply(sdme_ctx* ctx, const double* x_dev, double* y_dev);

/*
 * y_dev = (b1 M + K_T(u)) x_dev, the effective tangent of eq. NR_explicit
 * (consistent linearisation, Sec. 3, eq. effective stiffness 2), with the
 * rows and columns of constrained DOFs replaced by the identity.  Arithmetic
 * in the context's precision (float32 contractions for SDME_MIXED_FP32).
 */
sdme_status sdme_tangent_apply(sdme_ctx* ctx, const double* u_dev, double b1, const double* x_dev,
                               double* y_dev);

/* d_dev = diag(b1 M + K_T(u)), 1 on constrained DOFs (Jacobi preconditioner of the CGD solver). */
sdme_status sdme_diagonal(sdme_ctx* ctx, const double* u_dev, double b1, double* d_dev);

/*
 * Solve (b1 M + K_T(u)) x = b (constrained rows identity, b's constrained
 * entries ignored and x's set to 0) by Jacobi-preconditioned CG from x = 0,
 * stopping when ||r||_2 <= rtol ||b||_2 (CGD of Sec. 5).  Writes the
 * iteration count and the final relative residual (host pointers, may be
 * NULL).  SDME_PCG_MAXIT when maxit is reached.
 * SDME_MIXED_FP32: the iterations run in float32 with the solution summed in
 * float64; when the float32 recurrence meets the test, the float64 residual
 * b - (b1 M + K_T(u)) x is formed with the float64 operator (the stored
 * float64 state) and the recurrence restarts from it until that residual
 * meets the test (iterative refinement; at most the restarts set by
 * sdme_set_refinement, each required to halve the residual).  final_rel is
 * then the float64 residual's.
 */
sdme_status sdme_pcg_solve(sdme_ctx* ctx, const double* u_dev, double b1, const double* b_dev,
                           double* x_dev, double rtol, int maxit, int* iters, double* final_rel);

/*
 * Dead uniform traction t[3] on face `face` (SDME_XMIN..SDME_ZMAX):
 * f_dev = int_face t . N_i dA (fourth term of eq. material virtual work).
 * Overwrites f_dev (device, ndof).  Host-side quadrature, one upload.
 */
sdme_status sdme_traction_load(sdme_ctx* ctx, int face, const double t[3], double* f_dev);

/*
 * Static condensation of the element-interior modes (the paper's solver
 * shape: Schur complement on the tangent matrix and residual, Sec. 4 and
 * Sec. 5.1).  When enabled, every effective-operator solve (sdme_pcg_solve,
 * the Newton iterations of sdme_implicit_newmark_step and sdme_static_solve)
 * forms the dense element matrices, factors their interior blocks
 * (Cholesky), builds the element Schur complements S_e = A_BB - A_BI A_II^-1
 * A_IB, runs Jacobi-PCG (diagonal of S) on the skeleton DOFs and recovers
 * the interior DOFs; iteration counts then refer to the condensed system.
 * Interior DOFs: lattice points none of whose indices is a multiple of P.
 * Memory: nelem (N^2 + Ni^2 + Ni Nb + Nb^2) float64 words, N = 3 (P+1)^3,
 * Ni = 3 (P-1)^3, Nb = N - Ni (about 67 MB per element at P = 8, 1.7 MB at
 * P = 4).  Float64 contexts only, P >= 2, at most 65535 elements, not for
 * SDME_NODAL_LUMPED (else SDME_EUNSUPPORTED); SDME_ENOMEM if the buffers do
 * not fit.  enable = 0 returns to the uncondensed path (buffers are kept).
 */
sdme_status sdme_set_condensation(sdme_ctx* ctx, int enable);

/*
 * Static equilibrium R(u) = P by Newton-Raphson without inertia (the static
 * problem of Sec. 5.1): psi = P - R(u), K_T(u) du = psi by Jacobi-PCG (rtol
 * pcg_rtol in FP64, mixed_rtol in MIXED_FP32), u += du, until
 * ||psi|| <= newton_tol max(||psi_0||, 1e-14 ||P||) or max_newton
 * iterations.  u_dev: initial guess in, solution out (constrained entries
 * are kept; the last iterate when the test is not met).  opts may be NULL (tol 1e-8, 50 iterations, pcg_rtol 1e-12);
 * beta and gamma are ignored.  Returns SDME_OK when converged,
 * SDME_NEWTON_DIVERGED otherwise, or the inner solver's failure.
 * Synchronises.
 */
sdme_status sdme_static_solve(sdme_ctx* ctx, double* u_dev, const double* P_dev, const sdme_newton_opts* opts,
                              sdme_step_stats* stats);

/*
 * One implicit Newmark step t_n -> t_{n+1} solved by Newton-Raphson with
 * Jacobi-PCG linear solves (Sec. 4.2, eqs. Eq:residual, NR_explicit):
 *   psi = P_{n+1} - R(u^k) - M a(u^k),  a(u) = b1 (u - u_n) - b2 v_n - b3 a_n,
 *   (b1 M + K_T(u^k)) du = psi,  u^{k+1} = u^k + du,
 * predictor u^0 = u_n; then a_{n+1} and v_{n+1} by the Newmark formulas.
 * P_next_dev: external load at t_{n+1} (device, ndof).  Constrained entries of
 * state->u keep their values.  opts NULL selects defaults
 * (0.25, 0.5, 1e-8, 30, 1e-10, 1e-4, 20000).  stats may be NULL.
 * Returns SDME_OK when the Newton test is met.  Otherwise (SDME_NEWTON_DIVERGED
 * after max_newton iterations, SDME_NONPOSITIVE_J, SDME_NAN or the inner
 * solver's failure) the state is left at t_n: u is restored to u_n and v, a
 * are not touched; stats describe the failed attempt.
 */
sdme_status sdme_implicit_newmark_step(sdme_ctx* ctx, sdme_state* state, double dt,
                                       const double* P_next_dev, const sdme_newton_opts* opts,
                                       sdme_step_stats* stats);

/* State of the explicit central-difference scheme (device vectors, ndof each). */
typedef struct {
  double* u;             /* u_n (in) -> u_{n+1} (out); the call swaps u and u_prev */
  double* u_prev;        /* u_{n-1} (in) -> u_n (out) */
  double* a;             /* a_n = M^{-1} (P_n - R(u_n)) (out) */
} sdme_explicit_state;

/*
 * Start-up of the explicit central-difference scheme (Sec. 4.1):
 * a_0 = M^{-1} (P_0 - R(u_0)) by Jacobi-PCG on the consistent mass (rtol,
 * maxit), and u_{-1} = u_0 - dt v_0 + dt^2/2 a_0 written to state->u_prev
 * (constrained DOFs: u_{-1} = u_0).  state->u holds u_0 on entry.
 */
sdme_status sdme_explicit_start(sdme_ctx* ctx, sdme_explicit_state* state, double dt, const double* P0_dev,
                                const double* v0_dev, double rtol, int maxit);

/*
 * One explicit central-difference step (Sec. 4.1, eq. Motion_explicit2):
 * M a_n = P_n - R(u_n) solved by Jacobi-PCG on the consistent mass (rtol
 * relative, from zero), u_{n+1} = 2 u_n - u_{n-1} + dt^2 a_n on free DOFs.
 * The new displacement is written over u_{n-1} and the two pointers in
 * `state` are swapped, so state->u is u_{n+1} on return.  The mass solve
 * runs in the context's precision (float32 vectors for SDME_MIXED_FP32);
 * the residual and the state update are float64.  pcg_iters may be NULL.
 */
sdme_status sdme_explicit_step(sdme_ctx* ctx, sdme_explicit_state* state, double dt, const double* Pn_dev,
                               double rtol, int maxit, int* pcg_iters);

/*
 * Differentiating an explicit trajectory (the central-difference scheme of
 * Sec. 4.1, as in sdme_explicit_start / sdme_explicit_step) with respect to
 * the material constants (mu, lambda), the initial state and the load.
 *
 * A tape holds checkpoints (u_n, u_{n-1}) every `every` steps, a segment
 * buffer of `every` vectors for recomputation, and work vectors: about
 * (2 ceil(nsteps/every) + every + 10) float64 vectors of ndof entries,
 * owned by the tape.  It is bound to one context (used on its stream).
 */
typedef struct sdme_tape sdme_tape;

sdme_status sdme_tape_create(sdme_ctx* ctx, int nsteps, int every, sdme_tape** out);
sdme_status sdme_tape_destroy(sdme_tape* tape);

/*
 * Forward run recorded on the tape: start-up from (u0, v0) with P_0, then
 * nsteps explicit steps n = 0 .. nsteps-1 with loads P_n = s_host[n] * f_dev
 * (f_dev NULL: no load; s_host then unused, else nsteps host doubles).
 * Every mass solve is Jacobi-PCG to rtol (maxit iterations at most).
 * Writes u_N (N = nsteps) to uN_dev.  u0_dev, v0_dev, f_dev, uN_dev: float64
 * device vectors of ndof entries, caller-owned (f is copied into the tape).
 * Synchronises.
 */
sdme_status sdme_explicit_forward(sdme_ctx* ctx, sdme_tape* tape, double dt, const double* u0_dev,
                                  const double* v0_dev, const double* f_dev, const double* s_host, double rtol,
                                  int maxit, double* uN_dev);

/*
 * Discrete adjoint of the last sdme_explicit_forward on the tape for an
 * objective J(u_N), given gN_dev = dJ/du_N.  With A the mass inverse on the
 * free DOFs and z_n = A g_{n+1}, the sweep runs n = N-1 .. 0:
 *   g_n = [2 g_{n+1} - g_{n+2} on free DOFs | g_{n+1} on constrained] - dt^2 K_T(u_n) z_n,
 *   dJ/d(mu, lambda) -= dt^2 z_n . dR(u_n)/d(mu, lambda),  dJ/df += dt^2 s_n z_n,
 * then the start-up adjoint (g_{-1} = -g_1 on free DOFs, weight dt^2 / 2).
 * Segments between checkpoints are recomputed forward once each.  Outputs,
 * each optional (NULL): gmu, glambda (host doubles), gu0_dev, gv0_dev, gf_dev
 * (float64 device vectors, overwritten).  The context's material must be the
 * one of the forward run.  Synchronises.
 */
sdme_status sdme_explicit_adjoint(sdme_ctx* ctx, sdme_tape* tape, const double* gN_dev, double* gmu,
                                  double* glambda, double* gu0_dev, double* gv0_dev, double* gf_dev);

/*
 * Kinetic energy 1/2 v^T M v and strain energy int Psi(F(u)) dV (eq.
 * hyperelastic strain energy); either output may be NULL (its input may
 * then be NULL too).  Float64, synchronises.
 */
sdme_status sdme_energy(sdme_ctx* ctx, const double* u_dev, const double* v_dev, double* kinetic, double* strain);

/*
 * Critical explicit time step of the linearisation at u: power iteration on
 * M^{-1} K_T(u) (iters iterations, Rayleigh quotient, constrained DOFs
 * excluded) gives lambda_max; dt_crit = 2 / sqrt(lambda_max) (the central-
 * difference stability limit).  Either output may be NULL.
 */
sdme_status sdme_estimate_dt_crit(sdme_ctx* ctx, const double* u_dev, int iters, double* dt_crit,
                                  double* lambda_max);

/*
 * Body load f_dev = int N_i f dV (third term of eq. material virtual work,
 * f per unit reference volume) from f sampled at the Gauss points:
 * fq_dev[(e*3 + c)*Q^3 + q], element e = (ez ny + ey) nx + ex, component c,
 * Gauss point q = (k3 Q + k2) Q + k1 at reference coordinates
 * (xq[k1], xq[k2], xq[k3]) (sdme_gauss_points), Q = P + 2.  Overwrites f_dev.
 */
sdme_status sdme_body_load(sdme_ctx* ctx, const double* fq_dev, double* f_dev);

/*
 * Solve M x = b (consistent mass, constrained rows identity, b's constrained
 * entries ignored) by Jacobi-PCG from zero to ||r|| <= rtol ||b||, in the
 * context's precision; e.g. the L2 projection of an initial field.
 */
sdme_status sdme_mass_solve(sdme_ctx* ctx, const double* b_dev, double* x_dev, double rtol, int maxit, int* iters,
                            double* final_rel);

/* The context's Q = P + 2 Gauss-Legendre points and weights on [-1, 1] (host arrays, may be NULL). */
sdme_status sdme_gauss_points(const sdme_ctx* ctx, double* xq, double* wq);

/*
 * Physical coordinates of the Gauss points (the affine map of each box
 * element, eq. ProdTensorialHexaedro with the trilinear geometry):
 * X_dev[(e Q^3 + q) 3 + d], e and q ordered as for sdme_body_load; a
 * float64 device array of nelem Q^3 3 entries, caller-owned, overwritten.
 * Stream-ordered, no synchronisation.  SDME_EUNSUPPORTED for 2D contexts.
 */
sdme_status sdme_gauss_point_coords(sdme_ctx* ctx, double* X_dev);

/* Cumulative device event timings of the context (ms) and counts, for measurement. */
typedef struct {
  double tangent_ms;     /* sum of timed tangent-kernel launches */
  int64_t tangent_launches;
  int64_t kernel_launches; /* all kernels launched by this context */
} sdme_timing;

/* Description of the last CUDA runtime error the context met (after SDME_ECUDA). */
const char* sdme_cuda_error_string(const sdme_ctx* ctx);

/* Enable (1) / disable (0) CUDA-event timing of every tangent-kernel launch. */
sdme_status sdme_set_timing(sdme_ctx* ctx, int enable);
sdme_status sdme_get_timing(sdme_ctx* ctx, sdme_timing* out);

/*
 * MIXED_FP32 contexts: the largest number of float64-residual restarts
 * (iterative refinement) of one float32 PCG solve; 0 turns the refinement
 * off (the float32 recurrence's own test ends the solve).  Default 8.
 * Applies to the tangent solves (Newton steps, sdme_pcg_solve); mass solves
 * (explicit steps, sdme_mass_solve) end on the float32 recurrence's test.
 * Ignored by FP64 contexts.
 * SDME_EINVAL for a negative count.
 */
sdme_status sdme_set_refinement(sdme_ctx* ctx, int max_restarts);

/*
 * Launch shape of the tangent operator inside PCG (hexahedral meshes):
 * ctas = 0 one CTA per element (the default); ctas = -1 as many CTAs as fit
 * on the GPU at once (resident CTAs per SM x SMs); ctas > 0 that many.  With
 * a fixed grid each CTA serves elements blockIdx, blockIdx + grid, ..., and
 * sums its share of p.(A p) over them in that order (results stay
 * deterministic).  Drops the captured PCG graph.  SDME_EINVAL for ctas < -1.
 * sdme_get_tangent_grid returns the grid in use (0: one CTA per element).
 */
sdme_status sdme_set_tangent_grid(sdme_ctx* ctx, int ctas);
int sdme_get_tangent_grid(const sdme_ctx* ctx);

/*
 * y_dev = (b1 M + K_T(u)) x_dev in float64, like sdme_tangent_apply, but
 * without a context and without allocating anything: no cudaMalloc,
 * cudaFree, host heap or library allocation.  The paper has no counterpart;
 * this exists for callers that cannot allocate device memory, such as code
 * running under a fixed memory budget or a pool that forbids new device
 * allocations, or while other work must not be disturbed by allocator
 * synchronisation.
 *
 * Inputs: a hexahedral mesh, material and order P (1..8) as for
 * sdme_create (three-dimensional meshes only: nelem[2] = 0 returns
 * SDME_EINVAL); the 1D tables xq[Q], wq[Q], B[Q*(P+1)], D[Q*(P+1)] with
 * Q = P + 2, exactly as sdme_build_basis1d returns them (host arrays, read
 * during the call); u_dev (linearisation point), x_dev, y_dev: float64
 * device vectors of length 3 Nn.  Constrained DOFs get y = x, as in
 * sdme_tangent_apply.
 *
 * Scratch: the linearisation state and the discarded internal-force vector
 * live in one static device array of 2^21 float64 words (16 MiB) that every
 * GPU loading the library holds until the process exits.  A call needs
 * 32 + 3 Nn + 10 (P+2)^3 nelem words; larger problems return SDME_EINVAL.
 * The array is shared by all calls and keeps the last call's contents; the
 * call clears what must start at zero.  Calls that overlap on the GPU (for
 * example on two streams at once) race on the array and must be avoided.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for later
 * calls on that device; make that first call before any stream capture.
 * The kept address assumes that the device's context lives as long as the
 * process: after a cudaDeviceReset the array must be looked up again, which
 * this entry point does not do.  The call synchronises `stream` (NULL =
 * legacy default stream) to report SDME_NONPOSITIVE_J.
 */
sdme_status sdme_tangent_apply_noalloc(const sdme_mesh_desc* mesh, const sdme_material* mat, int P,
                                       const double* xq, const double* wq, const double* B, const double* D,
                                       const double* u_dev, double b1, const double* x_dev, double* y_dev,
                                       void* stream);

/*
 * Batches of independent problems (many meshes of uneven size, order and
 * material solved together).  Each problem is a box mesh with its own
 * order P (1..8) and material; the basis kind and its parameters are common
 * (the P of `basis` is ignored).  Global vectors of all problems are
 * concatenated: problem i's float64 vector (layout as for a context,
 * [3][Nz][Ny][Nx]) starts at offset off[i] of a buffer of total_len entries
 * (sdme_batch_layout); entries between segments are padding, kept zero.
 *
 * Every batched operation runs one launch per order group and step (not
 * one per problem): the element kernels take up to 128 problems per launch
 * with their scalars in the kernel parameter block, the per-DOF kernels
 * split the grid among the problems, and PCG keeps one scalar block per
 * problem so that each problem converges on its own; the PCG iterations are
 * replayed in chunks as one captured CUDA graph for the whole batch.
 */
typedef struct {
  sdme_mesh_desc mesh;
  sdme_material mat;
  int P;
} sdme_problem;

typedef struct sdme_batch sdme_batch;

/* stream: as for sdme_create.  SDME_EUNSUPPORTED if the basis lacks the
 * mirror symmetry (see sdme_create); SDME_EINVAL for invalid descriptors. */
sdme_status sdme_batch_create(sdme_batch** out, const sdme_problem* probs, int nprob, const sdme_basis_desc* basis,
                              sdme_precision prec, void* cuda_stream);
sdme_status sdme_batch_destroy(sdme_batch* b);

/* total_len: entries of a concatenated vector; off[i], ndof[i] (nprob each,
 * either may be NULL): segment offset and DOF count of problem i. */
sdme_status sdme_batch_layout(const sdme_batch* b, int64_t* total_len, int64_t* off, int64_t* ndof);

/* As sdme_internal_force / sdme_tangent_apply / sdme_traction_load, for
 * every problem at once.  t_host: 3 * nprob traction components (problem
 * i's traction at t_host[3 i]).  Synchronise. */
sdme_status sdme_batch_internal_force(sdme_batch* b, const double* u_dev, double* R_dev);
sdme_status sdme_batch_tangent_apply(sdme_batch* b, const double* u_dev, double b1, const double* x_dev,
                                     double* y_dev);
sdme_status sdme_batch_traction_load(sdme_batch* b, int face, const double* t_host, double* f_dev);

/*
 * One implicit Newmark step of every problem (as sdme_implicit_newmark_step,
 * same options for all; the inner tolerance is the fixed one, forcing is
 * ignored).  Each problem runs its own Newton iteration and
 * stops at its own tolerance; a problem that meets det F <= 0 or a PCG
 * breakdown stops there while the others continue.  stats (nprob entries,
 * may be NULL) receive each problem's record (converged = 0 for a problem
 * that failed).  Returns SDME_OK when every problem converged, else the
 * status of the first failing problem.
 */
sdme_status sdme_batch_newmark_step(sdme_batch* b, sdme_state* state, double dt, const double* P_next_dev,
                                    const sdme_newton_opts* opts, sdme_step_stats* stats);

/*
 * Launch-configuration tuner: for each order group, times the tangent
 * launch (the PCG's dominant kernel) on the batch's own problems, reps
 * launches per candidate, over one CTA per element and persistent grids of
 * 1, 2 and 4 CTAs per SM times the kernel's resident CTAs per SM, and keeps
 * the fastest for that order (for all element kernels of the group).  Needs
 * a linearisation state (call after any batched residual, tangent apply or
 * step).  orders/grids/ms (ngroups_max entries each, may be NULL) receive
 * each group's order, chosen grid (0 = one CTA per element) and time per
 * launch; *ngroups the number of groups.
 * Unless the persistent form is switched off (sdme_batch_set_persistent),
 * the tuner then times the PCG operator as one persistent launch across
 * all order groups: for each order the number of elements a work item
 * holds (1 up to 4, as many as 320 threads allow: one group of
 * 3 (P+2)^2 threads, rounded up to whole warps, per element), then the
 * whole batch with those tiles, and keeps the persistent launch for the
 * PCG iterations when it beats the sum of the per-order launches.
 */
sdme_status sdme_batch_tune(sdme_batch* b, int reps, int ngroups_max, int* ngroups, int* orders, int* grids,
                            float* ms);

/*
 * The PCG operator of a batch as one persistent launch across all order
 * groups (the benchmark spec's batching form): CTAs of 320 threads claim work items
 * (up to kper[P] consecutive elements of one problem of order P, one group
 * of threads per element) from a device counter until none is left; each
 * problem's last element to finish sums the problem's step-length partials.
 * No CTA waits on another.  mode: 1 always, 0 never (one launch per order
 * group), -1 (the default) as sdme_batch_tune decides, and then only while
 * problems of at least two orders are running.  kper (host, 9
 * entries indexed by P, may be NULL to keep the current ones): elements per
 * work item for each order, 1 up to min(4, 320 / threads per element)
 * (threads per element: 3 (P+2)^2 rounded up to a multiple of 32), else
 * SDME_EINVAL; the tuner overwrites them.  Setting the mode drops the
 * captured PCG graph.  SDME_EINVAL for another mode.
 */
sdme_status sdme_batch_set_persistent(sdme_batch* b, int mode, const int* kper);

/*
 * The persistent form's state: *on (1 when the PCG iterations may use it;
 * with mode -1 they do while at least two orders have running problems,
 * one order running being that order's single launch), kper[9] (elements
 * per work item by order, index = P), the tuner's time of one persistent
 * launch over the whole batch, the sum of the per-order launch times and
 * order_ms[9] (the persistent launch over one order's problems at its
 * chosen tile) (ms, -1 before tuning).  Any pointer may be NULL.
 */
sdme_status sdme_batch_persistent_info(const sdme_batch* b, int* on, int kper[9], float* persist_ms,
                                       float* groups_ms, float order_ms[9]);

/* Kernel launches issued by the batch so far (all kinds). */
sdme_status sdme_batch_launches(const sdme_batch* b, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* SDME_H */
