// C ABI of the engine: context set-up, the public operators, Jacobi-PCG and
// the Newton-Newmark driver.  All device work goes through the element
// kernels (elem_p<P>.cu) and the per-DOF kernels (vec_kernels.cuh).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/sdme.h"
#include "basis1d.h"
#include "common.cuh"
#include "elem_launch.h"
#include "cond_dense.cuh"
#include "eo_tables.h"
#include "vec_kernels.cuh"

using namespace sdme;

namespace {

constexpr int kVecBlocks = 152 * 8;      // per-DOF grid: 8 CTAs of 256 threads per SM
constexpr int kPcgChunk = 16;            // iterations per CUDA graph / host status read
// Up to this many elements the PCG step length is summed by the update
// kernel from the operator's per-element partials (every update CTA reads
// them all) instead of by the operator's last CTA.
constexpr int64_t kDeferMaxElems = 8192;

#define SDME_CUDA(call)                                           \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) {                                      \
      ctx->last_cuda = e_;                                        \
      return SDME_ECUDA;                                          \
    }                                                             \
  } while (0)

#define SDME_TRY(call)              \
  do {                              \
    sdme_status s_ = (call);        \
    if (s_ != SDME_OK) return s_;   \
  } while (0)

// NVTX range over a host scope (phases of a solve, seen by nsys / ncu
// --nvtx when a tool is attached; a no-op otherwise).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// Physical coordinates of the Gauss points, [nelem][Q^3][3].
struct GaussCoordParams {
  double xq[16];
  double h[3];
  int ne[3];
  int Q;
};

__global__ void k_gauss_coords(GaussCoordParams p, int64_t total, double* __restrict__ X) {
  const int Q3 = p.Q * p.Q * p.Q;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / Q3;
    const int q = (int)(i - e * Q3);
    const int k1 = q % p.Q, k2 = (q / p.Q) % p.Q, k3 = q / (p.Q * p.Q);
    const int ex = (int)(e % p.ne[0]), ey = (int)((e / p.ne[0]) % p.ne[1]), ez = (int)(e / ((int64_t)p.ne[0] * p.ne[1]));
    X[3 * i + 0] = p.h[0] * (ex + 0.5 * (1.0 + p.xq[k1]));
    X[3 * i + 1] = p.h[1] * (ey + 0.5 * (1.0 + p.xq[k2]));
    X[3 * i + 2] = p.h[2] * (ez + 0.5 * (1.0 + p.xq[k3]));
  }
}

}  // namespace

struct sdme_ctx {
  sdme_mesh_desc mesh{};
  sdme_material mat{};
  sdme_basis_desc basis{};
  sdme_precision prec = SDME_FP64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaError_t last_cuda = cudaSuccess;

  HostElemData h;
  MeshInfo mi{};
  int64_t ndof = 0;
  int Q = 0;

  // device buffers
  double* st64 = nullptr;
  float* st32 = nullptr;
  int* err = nullptr;
  PcgScalars* scal = nullptr;
  double* partial = nullptr;    // per-element / per-CTA partial sums
  int64_t upart_off = 0;        // PCG update partials start here (after the per-element ones)
  int* loc = nullptr;           // tangent gather / scatter offset table (3 n^3), or null
  // grids of the PCG update / direction kernels: one resident wave each
  // (index 0: float64 vectors, 1: float32), so the update's step-length
  // preamble runs once per SM slot
  int upd_blocks[2] = {kVecBlocks, kVecBlocks}, dir_blocks[2] = {kVecBlocks, kVecBlocks};
  double* dscal = nullptr;      // [0]: norm^2 results ; counters follow
  unsigned int* dcount = nullptr;
  // PCG vectors (x64: the solution of a float64 solve; in a MIXED_FP32
  // context x64, r64 and q64 hold the refinement's float64 solution,
  // residual and operator product)
  double *r64 = nullptr, *p64 = nullptr, *q64 = nullptr, *d64 = nullptr, *x64 = nullptr;
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
  // MIXED_FP32: the float32 solution (xh32; with xl32 the pair hi + lo of
  // the unrefined mass solves)
  float *xh32 = nullptr, *xl32 = nullptr;
  // iterative refinement of the float32 PCG (MIXED_FP32): at most this many
  // restarts from the float64 residual per solve (0: off), and the outcome
  // of the last solve
  int refine_max = 8;
  // PCG kernels of a chunk launched as programmatic dependents of their
  // predecessors (each starts on the SMs its predecessor frees)
  bool pdl = true;
  // CTAs of the PCG's tangent launch: 0 one per element, else that many
  // CTAs serving every tan_grid-th element (sdme_set_tangent_grid)
  int tan_grid = 0;
  int last_sweeps = 0;
  double last_true_rel = -1.0;
  // Newton work vectors
  double *un = nullptr, *ahat = nullptr, *mhat = nullptr, *y = nullptr, *psi = nullptr, *du = nullptr;
  // lumped (diagonal) mass of SDME_NODAL_LUMPED contexts, else null
  double* mlump = nullptr;
  // static condensation of the element-interior modes (sdme_set_condensation)
  bool cond = false;
  int cN = 0, cNi = 0, cNb = 0;
  int *cIl = nullptr, *cBl = nullptr, *cerr = nullptr;
  int64_t *cgI = nullptr, *cgB = nullptr;
  double *cKe = nullptr, *cL = nullptr, *cW = nullptr, *cS = nullptr, *cY = nullptr, *cg = nullptr;
  // pinned host mirrors
  PcgScalars* scal_h = nullptr;
  double* dscal_h = nullptr;
  int* err_h = nullptr;

  // PCG runs on a private stream (graph capture is not possible on the
  // legacy default stream), ordered after and before the caller's stream
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t gexec[1] = {nullptr};   // one chunk of PCG iterations (untimed mode)
  double gb1[1] = {0.0};
  int gop = 0;
  int gsize = 0;

  // measurement
  bool timing = false;
  int64_t timing_errors = 0;
  cudaError_t last_timing_error = cudaSuccess;
  double tangent_ms = 0.0;
  int64_t tangent_launches = 0;
  int64_t kernel_launches = 0;
  std::vector<cudaEvent_t> ev;
};

namespace {

template <typename F>
cudaError_t dispatch_P(int P, F&& f) {
  switch (P) {
    case 1: return f(std::integral_constant<int, 1>());
    case 2: return f(std::integral_constant<int, 2>());
    case 3: return f(std::integral_constant<int, 3>());
    case 4: return f(std::integral_constant<int, 4>());
    case 5: return f(std::integral_constant<int, 5>());
    case 6: return f(std::integral_constant<int, 6>());
    case 7: return f(std::integral_constant<int, 7>());
    case 8: return f(std::integral_constant<int, 8>());
    default: return cudaErrorInvalidValue;
  }
}

sdme_status check_basis(const sdme_basis_desc* b) {
  if (!b || b->P < 1 || b->P > kMaxP || b->kind < SDME_NODAL || b->kind > SDME_NODAL_LUMPED) return SDME_EINVAL;
  if (b->kind >= SDME_SDME_M && (b->k < 0.0 || b->k > 1.0)) return SDME_EINVAL;
  return SDME_OK;
}

// SDME_NODAL_LUMPED uses the nodal basis (only its mass treatment differs)
bool build_basis(const sdme_basis_desc* b, Basis1D& out) {
  const int kind = b->kind == SDME_NODAL_LUMPED ? (int)SDME_NODAL : (int)b->kind;
  return out.build(b->P, kind, b->k, b->lambda, b->start_nodal != 0, b->jacobi_alpha, b->jacobi_beta);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

sdme_status residual_launch(sdme_ctx* ctx, double b1, const double* u, double* y, bool with_state = true) {
  const HostElemData& h = ctx->h;
  float* st32 = (with_state && ctx->prec == SDME_MIXED_FP32) ? ctx->st32 : nullptr;
  double* st64 = with_state ? ctx->st64 : nullptr;
  SDME_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * ctx->ndof, ctx->stream));
  SDME_CUDA(dispatch_P(h.P, [&](auto Pc) {
    return launch_residual<decltype(Pc)::value>(h, b1, u, y, st64, st32, ctx->err, ctx->stream);
  }));
  ctx->kernel_launches += 1;
  return SDME_OK;
}

sdme_status sync_and_check(sdme_ctx* ctx) {
  SDME_CUDA(cudaMemcpyAsync(ctx->err_h, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  SDME_CUDA(cudaStreamSynchronize(ctx->stream));
  if (*ctx->err_h) {
    SDME_CUDA(cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream));
    return SDME_NONPOSITIVE_J;
  }
  return SDME_OK;
}

template <typename T, typename TV>
sdme_status tangent_launch(sdme_ctx* ctx, double b1, const TV* x, TV* y, double* partial, PcgScalars* scal,
                           cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr, bool defer = false, int grid = 0,
                           bool pdl = false) {
  const HostElemData& h = ctx->h;
  const T* st;
  if constexpr (sizeof(T) == 8) st = ctx->st64;
  else st = ctx->st32;
  if (e0) SDME_CUDA(cudaEventRecord(e0, ctx->stream));
  SDME_CUDA(dispatch_P(h.P, [&](auto Pc) {
    return launch_tangent<decltype(Pc)::value, T, TV>(h, b1, x, y, st, partial, scal, ctx->stream, defer, grid,
                                                      pdl && !e0);
  }));
  if (e1) SDME_CUDA(cudaEventRecord(e1, ctx->stream));
  ctx->kernel_launches += 1;
  return SDME_OK;
}

template <typename T>
sdme_status diag_launch(sdme_ctx* ctx, double b1, T* d, int inverse) {
  const HostElemData& h = ctx->h;
  const T* st;
  if constexpr (sizeof(T) == 8) st = ctx->st64;
  else st = ctx->st32;
  SDME_CUDA(cudaMemsetAsync(d, 0, sizeof(T) * ctx->ndof, ctx->stream));
  SDME_CUDA(dispatch_P(h.P, [&](auto Pc) {
    return launch_diag<decltype(Pc)::value, T>(h, b1, st, d, ctx->stream);
  }));
  k_diag_finish<T><<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, d, inverse);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 2;
  return SDME_OK;
}

// ||x||^2 on the host (synchronises)
sdme_status norm2_host(sdme_ctx* ctx, const double* x, double* out) {
  k_norm2<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->ndof, x, ctx->partial, ctx->dcount, ctx->dscal);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  SDME_CUDA(cudaMemcpyAsync(ctx->dscal_h, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  SDME_CUDA(cudaStreamSynchronize(ctx->stream));
  *out = ctx->dscal_h[0];
  return SDME_OK;
}

// Operators the PCG core can iterate on.
enum PcgOp { kOpTangent = 0, kOpMass = 1, kOpCondensed = 2 };

// Issue one chunk of PCG iterations (operator, update, direction) on ctx->stream.
template <typename T, typename TV>
sdme_status pcg_chunk(sdme_ctx* ctx, double b1, int op, bool tim, TV* r, TV* p, TV* q, TV* dinv, TV* xh, TV* xl) {
  // hexahedral tangent / mass operators leave p.(A p) as per-element (or,
  // with a fixed tangent grid, per-CTA) partials for the update kernel (no
  // last-CTA finalize in the operator)
  const int tgrid = (op == kOpTangent && ctx->h.dim == 3 && ctx->tan_grid > 0 && ctx->tan_grid < ctx->h.nelem)
                        ? ctx->tan_grid : 0;
  const int nparts = tgrid ? tgrid : (int)ctx->h.nelem;
  const bool defer = op != kOpCondensed && ctx->h.dim == 3 && nparts <= kDeferMaxElems;
  for (int j = 0; j < kPcgChunk; ++j) {
    if (op == kOpCondensed) {
      if constexpr (sizeof(TV) == 8) {
        if (tim) SDME_CUDA(cudaEventRecord(ctx->ev[2 * j], ctx->stream));
        cond_apply_kernel<<<ctx->h.nelem, 256, sizeof(double) * ctx->cNb, ctx->stream>>>(
            ctx->cNb, ctx->cgB, ctx->cS, p, q, ctx->partial, ctx->scal);
        if (tim) SDME_CUDA(cudaEventRecord(ctx->ev[2 * j + 1], ctx->stream));
        ctx->kernel_launches += 1;
      } else {
        return SDME_EUNSUPPORTED;
      }
    } else if (op == kOpMass) {
      SDME_CUDA(dispatch_P(ctx->h.P, [&](auto Pc) {
        return launch_mass_op<decltype(Pc)::value, T, TV>(ctx->h, b1, p, q, ctx->partial, ctx->scal, ctx->stream,
                                                          defer);
      }));
      ctx->kernel_launches += 1;
    } else {
      // the operator of every iteration after the chunk's first overlaps the
      // previous direction update's tail (programmatic dependent launch)
      SDME_TRY((tangent_launch<T, TV>(ctx, b1, p, q, ctx->partial, ctx->scal, tim ? ctx->ev[2 * j] : nullptr,
                                      tim ? ctx->ev[2 * j + 1] : nullptr, defer, tgrid, ctx->pdl && j > 0)));
    }
    // update and direction start while their predecessor drains (their CTAs
    // read the vectors the predecessor does not write before pdl_wait())
    constexpr int vi = sizeof(TV) == 4 ? 1 : 0;
    const bool pdl_vec = ctx->pdl && !tim;
    SDME_CUDA(launch_maybe_pdl(k_pcg_update<TV>, dim3(ctx->upd_blocks[vi]), dim3(kUpdThreads), 0, ctx->stream, pdl_vec,
                               ctx->ndof, r, q, (const TV*)dinv, ctx->scal, ctx->partial + ctx->upart_off,
                               (const double*)(defer ? ctx->partial : nullptr), nparts));
    SDME_CUDA(launch_maybe_pdl(k_pcg_direction<TV>, dim3(ctx->dir_blocks[vi]), dim3(kVecThreads), 0, ctx->stream,
                               ctx->pdl, ctx->ndof, (const TV*)r, (const TV*)dinv, p, xh, xl,
                               (const PcgScalars*)ctx->scal));
  }
  SDME_CUDA(cudaGetLastError());
  return SDME_OK;
}

// Runs the PCG body on the context's private stream: the private stream
// waits for the caller's stream on entry, and the caller's stream waits for
// the private stream on exit (also on error paths).
struct SideStreamScope {
  sdme_ctx* ctx;
  cudaStream_t user;
  explicit SideStreamScope(sdme_ctx* c) : ctx(c), user(c->stream) {
    cudaEventRecord(ctx->ev_fork, user);
    cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
    ctx->stream = ctx->side;
  }
  ~SideStreamScope() {
    cudaEventRecord(ctx->ev_join, ctx->side);
    cudaStreamWaitEvent(user, ctx->ev_join, 0);
    ctx->stream = user;
  }
};

// r64 = b - A x with the float64 operator (tangent with the stored float64
// state, or mass), zero on constrained DOFs; returns ||r64||^2 (synchronises).
sdme_status residual64(sdme_ctx* ctx, double b1, int op, const double* b, const double* x, double* rr) {
  SDME_CUDA(cudaMemsetAsync(ctx->q64, 0, sizeof(double) * ctx->ndof, ctx->stream));
  if (op == kOpMass) {
    SDME_CUDA(dispatch_P(ctx->h.P, [&](auto Pc) {
      return launch_mass_op<decltype(Pc)::value, double, double>(ctx->h, b1, x, ctx->q64, nullptr, nullptr,
                                                                 ctx->stream, false);
    }));
    ctx->kernel_launches += 1;
  } else {
    SDME_TRY((tangent_launch<double, double>(ctx, b1, x, ctx->q64, nullptr, nullptr)));
  }
  k_residual_combine<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, b, nullptr, ctx->q64, ctx->r64,
                                                                  ctx->partial, ctx->dcount, ctx->dscal);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  SDME_CUDA(cudaMemcpyAsync(ctx->dscal_h, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  SDME_CUDA(cudaStreamSynchronize(ctx->stream));
  *rr = ctx->dscal_h[0];
  return SDME_OK;
}

// Jacobi PCG on (b1 M + K_T) with the linearisation state already stored.
// b and x are float64 device vectors; the iteration runs in TV / T with the
// solution accumulated in xh (float64), in the float32 pair xh + xl (mass
// solves), or, for the refined float32 tangent solves, in a single float32 xh
// folded into the float64 x64 at every refinement check (xh then holds one
// sweep's correction only; 44 instead of 52 bytes of vector traffic per DOF
// and iteration, the pair's low word no longer read and written).  The iterations are issued in chunks
// of kPcgChunk captured once as a CUDA graph (kernels see the device-side
// status and return at once after convergence); the host reads the status
// between chunks.
// Float32 iterations are refined in float64: when the float32 recurrence
// meets the test, r = b - A x is formed with the float64 operator; while
// ||r|| > rtol ||b|| the recurrence restarts from r (at most refine_max
// times, and only while each restart at least halves ||r||).  The float32
// operator differs from the float64 one by about eps32 times the element-level
// magnitudes, which for smooth (low-eigenvalue) components is far above their
// assembled size; the restarts make the returned x meet the test with the
// float64 operator, as a float64 solve would.
template <typename T, typename TV>
sdme_status pcg_core(sdme_ctx* ctx, double b1, int op, const double* b, double* x, double rtol, int maxit,
                     int* iters, double* rel, TV* r, TV* p, TV* q, TV* dinv, TV* xh, TV* xl) {
  NvtxRange range_pcg("sdme pcg");
  SideStreamScope scope(ctx);
  if (op == kOpMass) {
    SDME_CUDA(cudaMemsetAsync(dinv, 0, sizeof(TV) * ctx->ndof, ctx->stream));
    SDME_CUDA(dispatch_P(ctx->h.P, [&](auto Pc) {
      return launch_mass_diag<decltype(Pc)::value, T>(ctx->h, b1, (T*)dinv, ctx->stream);
    }));
    k_diag_finish<T><<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, (T*)dinv, 1);
    SDME_CUDA(cudaGetLastError());
    ctx->kernel_launches += 2;
  } else if (op == kOpTangent) {
    NvtxRange range_diag("sdme diagonal");
    SDME_TRY(diag_launch<T>(ctx, b1, (T*)dinv, 1));
  }  // kOpCondensed: the caller has put 1 / diag(S) in dinv
  // mass solves are not refined: the consistent mass is well conditioned and
  // the explicit scheme's mixed tolerance (1e-6) is within float32 reach
  const bool refine = sizeof(TV) == 4 && ctx->refine_max > 0 && op == kOpTangent;
  if (refine) xl = nullptr;   // single float32 x per sweep, folded into x64 at each check
  bool folded = false;        // x64 holds the folded sweeps
  k_pcg_init<TV><<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, b, 1.0, dinv, xh, xl, r, p, q, ctx->scal,
                                                              ctx->partial, rtol, maxit);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  int done_iters = 0, sweeps = 0;
  double true_rel = -1.0;
  for (;;) {
    // launch accounting: one executed chunk = kPcgChunk x (operator, update,
    // direction); a capture issues launches that do not execute
    const int64_t l0 = ctx->kernel_launches;
    // Per-launch event timing needs the events recorded by plain stream
    // launches (events recorded inside a graph cannot be queried), so the
    // timed mode issues the chunk directly; the untimed mode replays a graph.
    const bool tim = ctx->timing;
    cudaGraphExec_t& ge = ctx->gexec[0];
    if (ge && (ctx->gb1[0] != b1 || ctx->gop != op || ctx->gsize != (int)sizeof(T))) {
      cudaGraphExecDestroy(ge);
      ge = nullptr;
    }
    NvtxRange range_chunk("sdme pcg chunk (operator, update, direction)");
    if (tim) {
      SDME_TRY((pcg_chunk<T, TV>(ctx, b1, op, true, r, p, q, dinv, xh, xl)));
    } else if (!ge) {
      // first chunk runs directly (also sets the kernels' attributes), then
      // the same chunk is captured for the following ones
      SDME_TRY((pcg_chunk<T, TV>(ctx, b1, op, false, r, p, q, dinv, xh, xl)));
      cudaGraph_t g = nullptr;
      SDME_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      sdme_status cs = pcg_chunk<T, TV>(ctx, b1, op, false, r, p, q, dinv, xh, xl);
      cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
      if (cs != SDME_OK) return cs;
      SDME_CUDA(ce);
      ce = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      SDME_CUDA(ce);
      ctx->gb1[0] = b1;
      ctx->gop = op;
      ctx->gsize = (int)sizeof(T);
    } else {
      SDME_CUDA(cudaGraphLaunch(ge, ctx->stream));
    }
    ctx->kernel_launches = l0 + 3 * kPcgChunk;
    SDME_CUDA(cudaMemcpyAsync(ctx->scal_h, ctx->scal, sizeof(PcgScalars), cudaMemcpyDeviceToHost, ctx->stream));
    SDME_CUDA(cudaStreamSynchronize(ctx->stream));
    const PcgScalars& s = *ctx->scal_h;
    if (tim) {
      // tangent launches of this chunk that ran with a live iteration: one per
      // completed iteration, plus the one that detected a breakdown
      int ran = s.iter - done_iters + (s.status == kPcgBreakdown ? 1 : 0);
      if (ran > kPcgChunk) ran = kPcgChunk;
      for (int j = 0; j < ran; ++j) {
        float ms = 0.f;
        const cudaError_t te = cudaEventElapsedTime(&ms, ctx->ev[2 * j], ctx->ev[2 * j + 1]);
        if (te == cudaSuccess) {
          ctx->tangent_ms += ms;
          ctx->tangent_launches += 1;
        } else {
          ctx->timing_errors += 1;
          ctx->last_timing_error = te;
          cudaGetLastError();  // the failed query must not surface at the next launch check
        }
      }
    }
    done_iters = s.iter;
    if (s.status == kPcgRunning) continue;
    if (s.status == kPcgConverged || s.status == kPcgMaxit) {
      // the last iteration's x += alpha p (its direction kernel returned at once)
      k_pcg_xfinal<TV><<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->ndof, p, xh, xl, ctx->scal);
      SDME_CUDA(cudaGetLastError());
      ctx->kernel_launches += 1;
    }
    if (refine && s.status == kPcgConverged) {
      double rr64 = 0.0;
      const double bb = s.bb;
      const int it = s.iter;
      {
        NvtxRange range_ref("sdme refinement residual (float64 operator)");
        k_pcg_xfold<TV><<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->ndof, xh, ctx->x64, folded ? 0 : 1);
        folded = true;
        SDME_CUDA(cudaGetLastError());
        ctx->kernel_launches += 1;
        SDME_TRY(residual64(ctx, b1, op, b, ctx->x64, &rr64));
      }
      const double prev = true_rel;
      true_rel = bb > 0.0 ? std::sqrt(rr64 / bb) : 0.0;
      if (!std::isfinite(true_rel)) return SDME_NAN;
      if (true_rel > rtol && sweeps < ctx->refine_max && it < maxit && (prev < 0.0 || true_rel <= 0.5 * prev)) {
        ++sweeps;
        k_pcg_restart<TV><<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, ctx->r64, dinv, r, p, q,
                                                                       ctx->scal, ctx->partial);
        SDME_CUDA(cudaGetLastError());
        ctx->kernel_launches += 1;
        continue;
      }
    }
    break;
  }
  const PcgScalars& s = *ctx->scal_h;
  if (iters) *iters = s.iter;
  ctx->last_sweeps = sweeps;
  ctx->last_true_rel = true_rel;
  if (rel) *rel = true_rel >= 0.0 ? true_rel : ((s.bb > 0.0) ? std::sqrt(s.rr / s.bb) : 0.0);
  if (folded) {
    k_pcg_xout64<TV><<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->ndof, xh, ctx->x64, x);
    SDME_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
  } else if ((void*)x != (void*)xh) {
    k_pcg_xout<TV><<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->ndof, xh, xl, x);
    SDME_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
  }
  if (s.status == kPcgBreakdown) return SDME_NAN;
  if (s.status == kPcgMaxit) return SDME_PCG_MAXIT;
  return SDME_OK;
}

sdme_status pcg_dispatch(sdme_ctx* ctx, double b1, const double* b, double* x, double rtol, int maxit,
                         int* iters, double* rel, bool mass_only = false) {
  const int op = mass_only ? kOpMass : kOpTangent;
  if (ctx->prec == SDME_MIXED_FP32)
    return pcg_core<float, float>(ctx, b1, op, b, x, rtol, maxit, iters, rel, ctx->r32, ctx->p32, ctx->q32,
                                  ctx->d32, ctx->xh32, ctx->xl32);
  return pcg_core<double, double>(ctx, b1, op, b, x, rtol, maxit, iters, rel, ctx->r64, ctx->p64, ctx->q64,
                                  ctx->d64, ctx->x64, nullptr);
}

// M x = b on the free DOFs (x = 0 on constrained ones): Jacobi-PCG on the
// consistent mass, or a division by the lumped mass of SDME_NODAL_LUMPED.
sdme_status mass_solve_core(sdme_ctx* ctx, const double* b, double* x, double rtol, int maxit, int* iters,
                            double* rel) {
  if (ctx->mlump) {
    k_lumped_solve<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, ctx->mlump, b, x);
    SDME_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
    if (iters) *iters = 0;
    if (rel) *rel = 0.0;
    return SDME_OK;
  }
  return pcg_dispatch(ctx, 1.0, b, x, rtol, maxit, iters, rel, true);
}

// (b1 M + K_T(u)) x = f through the Schur complement on the skeleton DOFs
// (linearisation state at u already stored): dense element matrices, their
// interior factorisation and element Schur complements, Jacobi-PCG on the
// condensed system, interior recovery.  Float64 contexts only.
sdme_status cond_solve(sdme_ctx* ctx, double b1, const double* f, double* x, double rtol, int maxit, int* iters,
                       double* rel) {
  const int ne = ctx->h.nelem, N = ctx->cN, Ni = ctx->cNi, Nb = ctx->cNb;
  cudaStream_t s = ctx->stream;
  SDME_CUDA(dispatch_P(ctx->h.P, [&](auto Pc) {
    return launch_cond_columns<decltype(Pc)::value>(ctx->h, b1, ctx->st64, ctx->cKe, s);
  }));
  SDME_CUDA(cudaMemsetAsync(ctx->cerr, 0, sizeof(int) * ne, s));
  cond_factor_kernel<<<ne, kCondThreads, 0, s>>>(N, Ni, ctx->cIl, ctx->cKe, ctx->cL, ctx->cerr);
  cond_trsm_kernel<<<ne, kCondThreads, 0, s>>>(N, Ni, Nb, ctx->cIl, ctx->cBl, ctx->cKe, ctx->cL, ctx->cW);
  const unsigned tiles = (unsigned)((Nb + 31) / 32);
  cond_syrk_kernel<<<dim3(tiles, tiles, ne), dim3(32, 32), 0, s>>>(N, Ni, Nb, ctx->cBl, ctx->cKe, ctx->cW, ctx->cS);
  SDME_CUDA(cudaGetLastError());
  // 1 / diag(S) (interior entries 1), condensed right-hand side
  SDME_CUDA(cudaMemsetAsync(ctx->d64, 0, sizeof(double) * ctx->ndof, s));
  cond_diag_kernel<<<ne, 256, 0, s>>>(Nb, ctx->cgB, ctx->cS, ctx->d64);
  cond_rhs_init<<<kVecBlocks, 256, 0, s>>>(ctx->mi, ctx->h.P, f, ctx->cg, ctx->d64);
  k_diag_finish<double><<<kVecBlocks, kVecThreads, 0, s>>>(ctx->mi, ctx->d64, 1);
  cond_rhs_kernel<<<ne, 256, sizeof(double) * Ni, s>>>(Ni, Nb, ctx->cgI, ctx->cgB, ctx->cL, ctx->cW, f, ctx->cg,
                                                       ctx->cY);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 9;
  std::vector<int> errs(ne);
  SDME_CUDA(cudaMemcpyAsync(errs.data(), ctx->cerr, sizeof(int) * ne, cudaMemcpyDeviceToHost, s));
  SDME_CUDA(cudaStreamSynchronize(s));
  for (int v : errs)
    if (v) return SDME_NAN;  // interior block not positive definite
  const sdme_status ps = pcg_core<double, double>(ctx, b1, kOpCondensed, ctx->cg, x, rtol, maxit, iters, rel,
                                                  ctx->r64, ctx->p64, ctx->q64, ctx->d64, ctx->x64, nullptr);
  if (ps != SDME_OK && ps != SDME_PCG_MAXIT) return ps;
  cond_recover_kernel<<<ne, 256, sizeof(double) * (Ni + Nb), s>>>(Ni, Nb, ctx->cgI, ctx->cgB, ctx->cL, ctx->cW,
                                                                  ctx->cY, x);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  return ps;
}

// The effective-operator solve of the Newton iteration and of sdme_pcg_solve.
sdme_status linear_solve(sdme_ctx* ctx, double b1, const double* f, double* x, double rtol, int maxit, int* iters,
                         double* rel) {
  if (ctx->cond) return cond_solve(ctx, b1, f, x, rtol, maxit, iters, rel);
  return pcg_dispatch(ctx, b1, f, x, rtol, maxit, iters, rel);
}

// Lumped mass of SDME_NODAL_LUMPED: rho detJ w_p w_q w_r (GLL weights) per
// element node, summed over the elements sharing the node; the same for the
// three components.
sdme_status build_lumped_mass(sdme_ctx* ctx) {
  const HostElemData& h = ctx->h;
  const int P = h.P, n = P + 1;
  std::vector<double> x(n), w(n);
  gauss_lobatto_legendre(P, x.data());
  gauss_lobatto_weights(P, x.data(), w.data());
  std::vector<double> m(ctx->ndof, 0.0);
  const double f = h.rho * h.detJ;
  for (int ez = 0; ez < h.ne[2]; ++ez)
    for (int ey = 0; ey < h.ne[1]; ++ey)
      for (int ex = 0; ex < h.ne[0]; ++ex)
        for (int r = 0; r < n; ++r)
          for (int q = 0; q < n; ++q)
            for (int p = 0; p < n; ++p) {
              const int64_t node = ((int64_t)(ez * P + r) * h.N[1] + (ey * P + q)) * h.N[0] + (ex * P + p);
              m[node] += f * w[p] * w[q] * w[r];
            }
  for (int c = 1; c < 3; ++c)
    for (int64_t i = 0; i < h.Nn; ++i) m[c * h.Nn + i] = m[i];
  SDME_CUDA(dalloc(&ctx->mlump, ctx->ndof));
  SDME_CUDA(cudaMemcpyAsync(ctx->mlump, m.data(), sizeof(double) * ctx->ndof, cudaMemcpyHostToDevice, ctx->stream));
  SDME_CUDA(cudaStreamSynchronize(ctx->stream));
  return SDME_OK;
}

// x . y (float64, deterministic), synchronises
sdme_status dot_host(sdme_ctx* ctx, const double* x, const double* y, double* out) {
  k_dot<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->ndof, x, y, ctx->partial, ctx->dcount, ctx->dscal);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  SDME_CUDA(cudaMemcpyAsync(ctx->dscal_h, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  SDME_CUDA(cudaStreamSynchronize(ctx->stream));
  *out = ctx->dscal_h[0];
  return SDME_OK;
}

void free_all(sdme_ctx* ctx) {
  void* dev[] = {ctx->st64, ctx->st32, ctx->err, ctx->scal, ctx->partial, ctx->dscal, ctx->dcount,
                 ctx->r64, ctx->p64, ctx->q64, ctx->d64, ctx->x64, ctx->r32, ctx->p32, ctx->q32, ctx->d32,
                 ctx->xh32, ctx->xl32,
                 ctx->un, ctx->ahat, ctx->mhat, ctx->y, ctx->psi, ctx->du, ctx->mlump,
                 ctx->cIl, ctx->cBl, ctx->cerr, ctx->cgI, ctx->cgB, ctx->cKe, ctx->cL, ctx->cW, ctx->cS,
                 ctx->cY, ctx->cg, ctx->loc};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (ctx->scal_h) cudaFreeHost(ctx->scal_h);
  if (ctx->dscal_h) cudaFreeHost(ctx->dscal_h);
  if (ctx->err_h) cudaFreeHost(ctx->err_h);
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  for (cudaGraphExec_t g : ctx->gexec)
    if (g) cudaGraphExecDestroy(g);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
}

}  // namespace

//-----------------------------------------------------------------------------
// Checkpointed explicit trajectory and its discrete adjoint.
//-----------------------------------------------------------------------------
struct sdme_tape {
  sdme_ctx* ctx = nullptr;
  int nsteps = 0, every = 0, nck = 0;
  double dt = 0.0, rtol = 0.0;
  int maxit = 0;
  bool have_f = false, ran = false;
  std::vector<double> s;     // load schedule, P_n = s[n] f
  double* f = nullptr;       // load shape (ndof)
  double* ck = nullptr;      // nck x 2 x ndof: (u_n, u_{n-1}) at n = k * every
  double* seg = nullptr;     // every x ndof: u_{n0} .. u_{n0 + every - 1} of the segment being reversed
  double* v[9] = {};         // u, u_prev, a, P_n, g_{n+2}, g_{n+1}, z, K z, adjoint right-hand side
};

namespace {

// P_n = s[n] f into the tape's load vector (zero without a load shape)
sdme_status tape_load(sdme_tape* tp, int n) {
  sdme_ctx* ctx = tp->ctx;
  if (tp->have_f) {
    k_to_double<double><<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->ndof, tp->f, tp->s[n], tp->v[3]);
    SDME_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
  } else {
    SDME_CUDA(cudaMemsetAsync(tp->v[3], 0, sizeof(double) * ctx->ndof, ctx->stream));
  }
  return SDME_OK;
}

sdme_status copy_vec(sdme_ctx* ctx, double* dst, const double* src) {
  SDME_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * ctx->ndof, cudaMemcpyDeviceToDevice, ctx->stream));
  return SDME_OK;
}

// z = A g (mass solve on the free DOFs), then K_T(u) z and the material
// partials; accumulates -c (w . dR/dmu, w . dR/dlambda) into gth and
// c s_n z into gf.
sdme_status adjoint_kernel_step(sdme_tape* tp, const double* u, const double* g, double c, double sn, double* gth,
                                double* gf) {
  sdme_ctx* ctx = tp->ctx;
  double* z = tp->v[6];
  double* Kz = tp->v[7];
  int its = 0;
  double rel = 0.0;
  SDME_TRY(mass_solve_core(ctx, g, z, tp->rtol, tp->maxit, &its, &rel));
  double pm = 0.0, pl = 0.0;
  SDME_TRY(sdme_internal_force_vjp(ctx, u, z, Kz, &pm, &pl));
  gth[0] -= c * pm;
  gth[1] -= c * pl;
  if (gf) {
    k_axpy<double><<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->ndof, c * sn, z, gf);
    SDME_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
  }
  return SDME_OK;
}

}  // namespace

// Newton-Raphson on psi(u) = P + mhat - (R(u) + b1 M u) = 0 (mhat may be
// null: no inertia), Jacobi-PCG inner solves on (b1 M + K_T(u)).  Updates u
// in place; fills st; returns the Newton outcome.
// Test: ||psi_k|| <= tol max(||psi_0||, ||P||), the paper's Newton tolerance
// (Sec. 5.1) read relative to the larger of the step's initial residual and
// the applied load.  A test relative to ||psi_0|| alone can fall below what
// float64 resolves: the residual of a displacement u is evaluated no better
// than about eps64 times the element-level forces of u, which grow with u
// while ||psi_0|| (one load increment) does not.
sdme_status newton_core(sdme_ctx* ctx, double* u, const double* P_next_dev, double b1, const double* mhat,
                        const sdme_newton_opts& o, sdme_step_stats& st) {
  const int64_t nd = ctx->ndof;
  cudaStream_t s = ctx->stream;
  double pn2 = 0.0;
  SDME_TRY(norm2_host(ctx, P_next_dev, &pn2));
  const double pnorm = std::sqrt(pn2);
  const double base_rtol = (ctx->prec == SDME_MIXED_FP32) ? o.mixed_rtol : o.pcg_rtol;
  double psi0 = -1.0, nrm_prev = -1.0, eta_prev = 0.01, ref = 0.0;
  sdme_status result = SDME_NEWTON_DIVERGED;
  for (int k = 0; k <= o.max_newton; ++k) {
    {
      NvtxRange range_res("sdme residual");
      SDME_TRY(residual_launch(ctx, b1, u, ctx->y));
    }
    k_residual_combine<<<kVecBlocks, kVecThreads, 0, s>>>(ctx->mi, P_next_dev, mhat, ctx->y, ctx->psi,
                                                        ctx->partial, ctx->dcount, ctx->dscal);
    SDME_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
    SDME_CUDA(cudaMemcpyAsync(ctx->dscal_h, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
    SDME_TRY(sync_and_check(ctx));
    const double nrm = std::sqrt(ctx->dscal_h[0]);
    if (!std::isfinite(nrm)) {
      result = SDME_NAN;
      break;
    }
    if (psi0 < 0.0) {
      psi0 = nrm;
      ref = std::max(psi0, pnorm);
    }
    if (k < 33) st.residuals[k] = nrm;
    st.residual_final = nrm;
    st.newton_iters = k;
    if (nrm <= o.newton_tol * ref) {
      result = SDME_OK;
      st.converged = 1;
      break;
    }
    if (k == o.max_newton) break;
    double inner_rtol = base_rtol;
    if (o.forcing == 1) {
      // Eisenstat-Walker forcing term (choice 2, gamma = 0.9, alpha = 2),
      // eta_0 = eta_max = 0.01
      double eta = 0.01;
      if (nrm_prev > 0.0) {
        const double ratio = nrm / nrm_prev;
        eta = 0.9 * ratio * ratio;
        const double safeguard = 0.9 * eta_prev * eta_prev;
        if (safeguard > 0.1) eta = std::max(eta, safeguard);
      }
      eta = std::min(eta, 0.01);
      eta = std::max(eta, 0.5 * o.newton_tol * ref / nrm);
      eta_prev = eta;
      inner_rtol = std::max(eta, base_rtol);
    }
    nrm_prev = nrm;
    int its = 0;
    double rel = 0.0;
    sdme_status ps = linear_solve(ctx, b1, ctx->psi, ctx->du, inner_rtol, o.pcg_maxit, &its, &rel);
    if (ps != SDME_OK && ps != SDME_PCG_MAXIT) {
      result = ps;
      break;
    }
    if (k < 32) st.pcg_iters[k] = its;
    st.pcg_iters_total += its;
    st.matvecs += its;
    st.refine_sweeps += ctx->last_sweeps;
    if (ctx->prec == SDME_MIXED_FP32 && !ctx->cond) st.lin_rel_max = std::max(st.lin_rel_max, rel);
    k_axpy<double><<<kVecBlocks, kVecThreads, 0, s>>>(nd, 1.0, ctx->du, u);
    SDME_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
  }
  st.residual0 = psi0;
  st.residual_ref = ref;
  return result;
}

extern "C" {

const char* sdme_status_string(sdme_status s) {
  switch (s) {
    case SDME_OK: return "ok";
    case SDME_EINVAL: return "invalid argument";
    case SDME_ENOMEM: return "out of memory";
    case SDME_ECUDA: return "CUDA runtime error";
    case SDME_PCG_MAXIT: return "PCG reached maxit";
    case SDME_NEWTON_DIVERGED: return "Newton did not converge";
    case SDME_NONPOSITIVE_J: return "non-positive Jacobian det F";
    case SDME_NAN: return "non-finite value";
    case SDME_TIMEOUT: return "device wait timed out";
    case SDME_EUNSUPPORTED: return "unsupported option";
  }
  return "unknown status";
}

sdme_status sdme_build_basis1d(const sdme_basis_desc* basis, int Q, double* xq, double* wq, double* B, double* D,
                               double* M1, double* K1) {
  if (check_basis(basis) != SDME_OK || Q < 1 || Q > 16) return SDME_EINVAL;
  Basis1D b;
  if (!build_basis(basis, b)) return SDME_EINVAL;
  std::vector<double> x(Q), w(Q);
  gauss_legendre(Q, x.data(), w.data());
  if (xq) std::memcpy(xq, x.data(), sizeof(double) * Q);
  if (wq) std::memcpy(wq, w.data(), sizeof(double) * Q);
  b.tables(Q, x.data(), B, D);
  if (M1 || K1) {
    std::vector<double> M, K;
    b.matrices(M, K, true);
    const int n = b.n;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const int pi = b.lattice_to_paper(i), pj = b.lattice_to_paper(j);
        if (M1) M1[i * n + j] = M[pi * n + pj];
        if (K1) K1[i * n + j] = K[pi * n + pj];
      }
  }
  return SDME_OK;
}

sdme_status sdme_create(sdme_ctx** out, const sdme_mesh_desc* mesh, const sdme_material* mat,
                        const sdme_basis_desc* basis, sdme_precision prec, void* stream) {
  if (!out || !mesh || !mat) return SDME_EINVAL;
  *out = nullptr;
  if (check_basis(basis) != SDME_OK) return SDME_EINVAL;
  if (prec != SDME_FP64 && prec != SDME_MIXED_FP32) return SDME_EINVAL;
  // nelem[2] == 0: a plane-strain mesh of quadrilaterals in the x-y plane
  const int dim = mesh->nelem[2] == 0 ? 2 : 3;
  for (int d = 0; d < dim; ++d)
    if (mesh->nelem[d] < 1 || mesh->nelem[d] > (1 << 24) || !(mesh->length[d] > 0.0) ||
        !std::isfinite(mesh->length[d]))
      return SDME_EINVAL;
  if (dim == 2 && (mesh->clamp[4] != 0 || mesh->clamp[5] != 0 || basis->kind == SDME_NODAL_LUMPED))
    return SDME_EINVAL;
  if (!(mat->mu > 0.0) || !(mat->lambda >= 0.0) || !(mat->rho >= 0.0) || !std::isfinite(mat->mu) ||
      !std::isfinite(mat->lambda) || !std::isfinite(mat->rho))
    return SDME_EINVAL;
  const int P = basis->P, n = P + 1, Q = P + 2;
  int64_t N[3];
  for (int d = 0; d < 3; ++d) N[d] = (d < dim) ? (int64_t)mesh->nelem[d] * P + 1 : 1;
  // element and DOF counts bounded in floating point first (no integer overflow)
  if ((double)mesh->nelem[0] * mesh->nelem[1] * (dim == 3 ? mesh->nelem[2] : 1) > 2147483647.0 ||
      3.0 * (double)N[0] * (double)N[1] * (double)N[2] > (double)((int64_t)1 << 40))
    return SDME_EINVAL;
  const int64_t nelem = (int64_t)mesh->nelem[0] * mesh->nelem[1] * (dim == 3 ? mesh->nelem[2] : 1);

  sdme_ctx* ctx = new (std::nothrow) sdme_ctx();
  if (!ctx) return SDME_ENOMEM;
  ctx->mesh = *mesh;
  ctx->mat = *mat;
  ctx->basis = *basis;
  ctx->prec = prec;
  Basis1D b;
  if (!build_basis(basis, b)) {
    delete ctx;
    return SDME_EINVAL;
  }
  HostElemData& h = ctx->h;
  h.P = P;
  h.nelem = (int)nelem;
  h.B.resize(Q * n);
  h.D.resize(Q * n);
  h.DQ.resize(Q * Q);
  h.W.resize(Q);
  std::vector<double> xq(Q);
  gauss_legendre(Q, xq.data(), h.W.data());
  b.tables(Q, xq.data(), h.B.data(), h.D.data());
  collocation_derivative(Q, xq.data(), h.DQ.data());
  {
    const EoSizes z(P);
    h.TE.resize(z.QH * z.NE);
    h.TO.resize(z.QH * z.NO);
    h.TEm.resize(z.NE);
    h.AH.resize(z.QH * z.QH);
    h.CH.resize(z.QH * z.QH);
    h.CM.resize(z.QH);
    h.DM.resize(z.QH);
    const int sym = build_eo_tables(P, h.B.data(), h.DQ.data(), h.TE.data(), h.TO.data(), h.TEm.data(),
                                    h.AH.data(), h.CH.data(), h.CM.data(), h.DM.data());
    if (sym == kEoNone) {  // e.g. a modal basis with jacobi_alpha != jacobi_beta
      delete ctx;
      return SDME_EUNSUPPORTED;
    }
    h.pairs = sym == kEoNodalPairs ? 1 : 0;
  }
  double hh[3];
  h.dim = dim;
  for (int d = 0; d < 3; ++d) {
    hh[d] = d < dim ? mesh->length[d] / mesh->nelem[d] : 2.0;
    h.s[d] = d < dim ? 2.0 / hh[d] : 0.0;
    h.ne[d] = d < dim ? mesh->nelem[d] : 1;
    h.N[d] = (int)N[d];
    ctx->mi.N[d] = (int)N[d];
  }
  h.detJ = dim == 3 ? hh[0] * hh[1] * hh[2] / 8.0 : hh[0] * hh[1] / 4.0;
  h.mu = mat->mu;
  h.lam = mat->lambda;
  h.rho = mat->rho;
  h.Nn = N[0] * N[1] * N[2];
  for (int f = 0; f < 6; ++f) h.clamp[f] = ctx->mi.clamp[f] = mesh->clamp[f] & 7u;
  ctx->mi.Nn = h.Nn;
  ctx->mi.ndof = dim * h.Nn;
  ctx->ndof = dim * h.Nn;
  ctx->Q = Q;

  // NULL is the legacy default stream, which orders with every other
  // blocking stream of the process (torch's default stream included).
  ctx->stream = (cudaStream_t)stream;
  ctx->own_stream = false;
  const int64_t nst = nelem * kStateFields * (int64_t)Q * Q * Q;
  const int64_t nd = ctx->ndof;
  ctx->upart_off = (nelem + 31) / 32 * 32;
  const int64_t npart = std::max<int64_t>(2 * nelem, 2 * kVecBlocks) + 64 + ctx->upart_off + 2 * kVecBlocks;
  bool ok = true;
  ok = ok && dalloc(&ctx->st64, nst) == cudaSuccess;
  if (prec == SDME_MIXED_FP32) ok = ok && dalloc(&ctx->st32, nst) == cudaSuccess;
  ok = ok && dalloc(&ctx->err, 1) == cudaSuccess;
  ok = ok && dalloc(&ctx->scal, 1) == cudaSuccess;
  ok = ok && dalloc(&ctx->partial, npart) == cudaSuccess;
  if (ok && dim == 3 && P % 2 == 0 && 3 * h.Nn <= (int64_t)INT32_MAX) {
    // offset of entry (c, r, q, p) from the element's corner lattice point
    std::vector<int> loc(3 * n * n * n);
    for (int c = 0; c < 3; ++c)
      for (int r = 0; r < n; ++r)
        for (int q = 0; q < n; ++q)
          for (int pp = 0; pp < n; ++pp)
            loc[((c * n + r) * n + q) * n + pp] = (int)(c * h.Nn + ((int64_t)r * h.N[1] + q) * h.N[0] + pp);
    ok = dalloc(&ctx->loc, (int64_t)loc.size()) == cudaSuccess &&
         cudaMemcpy(ctx->loc, loc.data(), sizeof(int) * loc.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    h.loc = ctx->loc;
  }
  ok = ok && dalloc(&ctx->dscal, 8) == cudaSuccess;
  ok = ok && dalloc(&ctx->dcount, 8) == cudaSuccess;
  if (prec == SDME_MIXED_FP32) {
    ok = ok && dalloc(&ctx->r32, nd) == cudaSuccess && dalloc(&ctx->p32, nd) == cudaSuccess &&
         dalloc(&ctx->q32, nd) == cudaSuccess && dalloc(&ctx->d32, nd) == cudaSuccess &&
         dalloc(&ctx->x64, nd) == cudaSuccess && dalloc(&ctx->r64, nd) == cudaSuccess &&
         dalloc(&ctx->q64, nd) == cudaSuccess && dalloc(&ctx->xh32, nd) == cudaSuccess &&
         dalloc(&ctx->xl32, nd) == cudaSuccess;
  } else {
    ok = ok && dalloc(&ctx->r64, nd) == cudaSuccess && dalloc(&ctx->p64, nd) == cudaSuccess &&
         dalloc(&ctx->q64, nd) == cudaSuccess && dalloc(&ctx->d64, nd) == cudaSuccess &&
         dalloc(&ctx->x64, nd) == cudaSuccess;
  }
  ok = ok && dalloc(&ctx->un, nd) == cudaSuccess && dalloc(&ctx->ahat, nd) == cudaSuccess &&
       dalloc(&ctx->mhat, nd) == cudaSuccess && dalloc(&ctx->y, nd) == cudaSuccess &&
       dalloc(&ctx->psi, nd) == cudaSuccess && dalloc(&ctx->du, nd) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&ctx->scal_h, sizeof(PcgScalars)) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&ctx->dscal_h, 8 * sizeof(double)) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&ctx->err_h, sizeof(int)) == cudaSuccess;
  if (ok) {
    ctx->ev.resize(2 * kPcgChunk);
    for (auto& e : ctx->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) == cudaSuccess;
  }
  if (ok) {
    ok = cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream) == cudaSuccess &&
         cudaMemsetAsync(ctx->scal, 0, sizeof(PcgScalars), ctx->stream) == cudaSuccess &&
         cudaMemsetAsync(ctx->dcount, 0, 8 * sizeof(unsigned int), ctx->stream) == cudaSuccess &&
         cudaStreamSynchronize(ctx->stream) == cudaSuccess;
  }
  if (ok) {
    int dev = 0, sms = 0;
    ok = cudaGetDevice(&dev) == cudaSuccess &&
         cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
    auto wave = [&](auto kernel, int* out, int threads = kVecThreads) {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess) return false;
      *out = std::max(1, std::min(kVecBlocks, per_sm * sms));
      return true;
    };
    ok = ok && wave(k_pcg_update<double>, &ctx->upd_blocks[0], kUpdThreads) &&
         wave(k_pcg_update<float>, &ctx->upd_blocks[1], kUpdThreads) &&
         wave(k_pcg_direction<double>, &ctx->dir_blocks[0]) && wave(k_pcg_direction<float>, &ctx->dir_blocks[1]);
  }
  if (ok && basis->kind == SDME_NODAL_LUMPED) ok = build_lumped_mass(ctx) == SDME_OK;
  if (!ok) {
    cudaGetLastError();
    free_all(ctx);
    delete ctx;
    return SDME_ENOMEM;
  }
  *out = ctx;
  return SDME_OK;
}

sdme_status sdme_destroy(sdme_ctx* ctx) {
  if (!ctx) return SDME_EINVAL;
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
  return SDME_OK;
}

sdme_status sdme_get_sizes(const sdme_ctx* ctx, int64_t* ndof, int N[3], int64_t* nelem) {
  if (!ctx) return SDME_EINVAL;
  if (ndof) *ndof = ctx->ndof;
  if (N)
    for (int d = 0; d < 3; ++d) N[d] = ctx->h.N[d];
  if (nelem) *nelem = ctx->h.nelem;
  return SDME_OK;
}

sdme_status sdme_internal_force(sdme_ctx* ctx, const double* u_dev, double* R_dev) {
  if (!ctx || !u_dev || !R_dev) return SDME_EINVAL;
  SDME_TRY(residual_launch(ctx, 0.0, u_dev, R_dev));
  return sync_and_check(ctx);
}

sdme_status sdme_set_material(sdme_ctx* ctx, const sdme_material* mat) {
  if (!ctx || !mat) return SDME_EINVAL;
  if (!(mat->mu > 0.0) || !(mat->lambda >= 0.0) || !(mat->rho >= 0.0)) return SDME_EINVAL;
  ctx->mat = *mat;
  ctx->h.mu = mat->mu;
  ctx->h.lam = mat->lambda;
  ctx->h.rho = mat->rho;
  // the captured PCG chunk holds the old parameter blocks
  for (cudaGraphExec_t& g : ctx->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  return SDME_OK;
}

sdme_status sdme_set_condensation(sdme_ctx* ctx, int enable) {
  if (!ctx) return SDME_EINVAL;
  if (!enable) {
    ctx->cond = false;
    return SDME_OK;
  }
  if (ctx->cond) return SDME_OK;
  const HostElemData& h = ctx->h;
  const int P = h.P, n = P + 1, n3 = n * n * n;
  if (ctx->prec != SDME_FP64 || ctx->mlump || P < 2 || h.nelem > 65535 || h.dim != 3) return SDME_EUNSUPPORTED;
  const int N = 3 * n3, Ni = 3 * (n - 2) * (n - 2) * (n - 2), Nb = N - Ni;
  std::vector<int> Il, Bl;
  for (int idx = 0; idx < N; ++idx) {
    const int m = idx % n3, p = m % n, q = (m / n) % n, r = m / (n * n);
    const bool inner = p > 0 && p < n - 1 && q > 0 && q < n - 1 && r > 0 && r < n - 1;
    (inner ? Il : Bl).push_back(idx);
  }
  const int ne = h.nelem;
  std::vector<int64_t> gI((size_t)ne * Ni), gB((size_t)ne * Nb);
  for (int e = 0; e < ne; ++e) {
    const int ex = e % h.ne[0], ey = (e / h.ne[0]) % h.ne[1], ez = e / (h.ne[0] * h.ne[1]);
    auto global = [&](int idx, bool* cons) {
      const int c = idx / n3, m = idx % n3, p = m % n, q = (m / n) % n, r = m / (n * n);
      const int ix = ex * P + p, iy = ey * P + q, iz = ez * P + r;
      const unsigned bit = 1u << c;
      *cons = (ix == 0 && (h.clamp[0] & bit)) || (ix == h.N[0] - 1 && (h.clamp[1] & bit)) ||
              (iy == 0 && (h.clamp[2] & bit)) || (iy == h.N[1] - 1 && (h.clamp[3] & bit)) ||
              (iz == 0 && (h.clamp[4] & bit)) || (iz == h.N[2] - 1 && (h.clamp[5] & bit));
      return c * h.Nn + ((int64_t)iz * h.N[1] + iy) * h.N[0] + ix;
    };
    bool cons;
    for (int i = 0; i < Ni; ++i) gI[(size_t)e * Ni + i] = global(Il[i], &cons);
    for (int b = 0; b < Nb; ++b) {
      const int64_t g = global(Bl[b], &cons);
      gB[(size_t)e * Nb + b] = cons ? -1 : g;
    }
  }
  bool ok = dalloc(&ctx->cIl, Ni) == cudaSuccess && dalloc(&ctx->cBl, Nb) == cudaSuccess &&
            dalloc(&ctx->cerr, ne) == cudaSuccess && dalloc(&ctx->cgI, (size_t)ne * Ni) == cudaSuccess &&
            dalloc(&ctx->cgB, (size_t)ne * Nb) == cudaSuccess &&
            dalloc(&ctx->cKe, (size_t)ne * N * N) == cudaSuccess &&
            dalloc(&ctx->cL, (size_t)ne * Ni * Ni) == cudaSuccess &&
            dalloc(&ctx->cW, (size_t)ne * Ni * Nb) == cudaSuccess &&
            dalloc(&ctx->cS, (size_t)ne * Nb * Nb) == cudaSuccess &&
            dalloc(&ctx->cY, (size_t)ne * Ni) == cudaSuccess && dalloc(&ctx->cg, ctx->ndof) == cudaSuccess;
  if (ok) {
    cudaStream_t s = ctx->stream;
    ok = cudaMemcpyAsync(ctx->cIl, Il.data(), sizeof(int) * Ni, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(ctx->cBl, Bl.data(), sizeof(int) * Nb, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(ctx->cgI, gI.data(), sizeof(int64_t) * gI.size(), cudaMemcpyHostToDevice, s) ==
             cudaSuccess &&
         cudaMemcpyAsync(ctx->cgB, gB.data(), sizeof(int64_t) * gB.size(), cudaMemcpyHostToDevice, s) ==
             cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    for (void* p : {(void*)ctx->cIl, (void*)ctx->cBl, (void*)ctx->cerr, (void*)ctx->cgI, (void*)ctx->cgB,
                    (void*)ctx->cKe, (void*)ctx->cL, (void*)ctx->cW, (void*)ctx->cS, (void*)ctx->cY, (void*)ctx->cg})
      if (p) cudaFree(p);
    ctx->cIl = ctx->cBl = ctx->cerr = nullptr;
    ctx->cgI = ctx->cgB = nullptr;
    ctx->cKe = ctx->cL = ctx->cW = ctx->cS = ctx->cY = ctx->cg = nullptr;
    return SDME_ENOMEM;
  }
  ctx->cN = N;
  ctx->cNi = Ni;
  ctx->cNb = Nb;
  ctx->cond = true;
  return SDME_OK;
}

sdme_status sdme_internal_force_vjp(sdme_ctx* ctx, const double* u_dev, const double* w_dev, double* gu_dev,
                                    double* gmu, double* glambda) {
  if (!ctx || !u_dev || !w_dev || !gu_dev) return SDME_EINVAL;
  if (ctx->h.dim != 3) return SDME_EUNSUPPORTED;
  SDME_TRY(residual_launch(ctx, 0.0, u_dev, ctx->y));
  SDME_CUDA(cudaMemsetAsync(gu_dev, 0, sizeof(double) * ctx->ndof, ctx->stream));
  SDME_CUDA(dispatch_P(ctx->h.P, [&](auto Pc) {
    return launch_vjp<decltype(Pc)::value>(ctx->h, w_dev, gu_dev, ctx->st64, ctx->partial, ctx->dcount,
                                           ctx->dscal, ctx->stream);
  }));
  ctx->kernel_launches += 1;
  SDME_CUDA(cudaMemcpyAsync(ctx->dscal_h, ctx->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  SDME_TRY(sync_and_check(ctx));
  if (gmu) *gmu = ctx->dscal_h[0];
  if (glambda) *glambda = ctx->dscal_h[1];
  return SDME_OK;
}

sdme_status sdme_mass_apply(sdme_ctx* ctx, const double* x_dev, double* y_dev) {
  if (!ctx || !x_dev || !y_dev) return SDME_EINVAL;
  if (ctx->mlump) {
    k_diag_mul<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->ndof, ctx->mlump, x_dev, y_dev);
    SDME_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
    return SDME_OK;
  }
  SDME_CUDA(cudaMemsetAsync(y_dev, 0, sizeof(double) * ctx->ndof, ctx->stream));
  SDME_CUDA(dispatch_P(ctx->h.P, [&](auto Pc) {
    return launch_mass<decltype(Pc)::value>(ctx->h, x_dev, y_dev, ctx->stream);
  }));
  ctx->kernel_launches += 1;
  return SDME_OK;
}

sdme_status sdme_tangent_apply(sdme_ctx* ctx, const double* u_dev, double b1, const double* x_dev, double* y_dev) {
  if (!ctx || !u_dev || !x_dev || !y_dev) return SDME_EINVAL;
  if (ctx->mlump && b1 != 0.0) return SDME_EUNSUPPORTED;
  SDME_TRY(residual_launch(ctx, 0.0, u_dev, ctx->y));
  SDME_TRY(sync_and_check(ctx));
  k_mask_init<double><<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, x_dev, y_dev);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  if (ctx->prec == SDME_MIXED_FP32) return tangent_launch<float, double>(ctx, b1, x_dev, y_dev, nullptr, nullptr);
  return tangent_launch<double, double>(ctx, b1, x_dev, y_dev, nullptr, nullptr);
}

sdme_status sdme_diagonal(sdme_ctx* ctx, const double* u_dev, double b1, double* d_dev) {
  if (!ctx || !u_dev || !d_dev) return SDME_EINVAL;
  if (ctx->mlump && b1 != 0.0) return SDME_EUNSUPPORTED;
  SDME_TRY(residual_launch(ctx, 0.0, u_dev, ctx->y));
  SDME_TRY(sync_and_check(ctx));
  return diag_launch<double>(ctx, b1, d_dev, 0);
}

sdme_status sdme_pcg_solve(sdme_ctx* ctx, const double* u_dev, double b1, const double* b_dev, double* x_dev,
                           double rtol, int maxit, int* iters, double* final_rel) {
  if (!ctx || !u_dev || !b_dev || !x_dev || maxit < 1 || !(rtol >= 0.0)) return SDME_EINVAL;
  if (ctx->mlump && b1 != 0.0) return SDME_EUNSUPPORTED;
  SDME_TRY(residual_launch(ctx, 0.0, u_dev, ctx->y));
  SDME_TRY(sync_and_check(ctx));
  return linear_solve(ctx, b1, b_dev, x_dev, rtol, maxit, iters, final_rel);
}

sdme_status sdme_traction_load(sdme_ctx* ctx, int face, const double t[3], double* f_dev) {
  if (!ctx || !t || !f_dev || face < 0 || face > 5) return SDME_EINVAL;
  const HostElemData& h = ctx->h;
  const int P = h.P, n = P + 1, Q = ctx->Q;
  if (h.dim == 2) {
    // dead traction (t[0], t[1]) on one edge of the rectangle (per unit out-of-plane length)
    if (face > 3) return SDME_EINVAL;
    std::vector<double> I(n, 0.0);
    for (int q = 0; q < Q; ++q)
      for (int j = 0; j < n; ++j) I[j] += h.W[q] * h.B[q * n + j];
    const int axis = face / 2, side = face % 2, tang = 1 - axis;
    const double jac = 0.5 * ctx->mesh.length[tang] / ctx->mesh.nelem[tang];
    const int fixed = side ? h.N[axis] - 1 : 0;
    std::vector<double> f(ctx->ndof, 0.0);
    for (int et = 0; et < h.ne[tang]; ++et)
      for (int a = 0; a < n; ++a) {
        int idx[2];
        idx[axis] = fixed;
        idx[tang] = et * P + a;
        const int64_t node = (int64_t)idx[1] * h.N[0] + idx[0];
        for (int c = 0; c < 2; ++c) f[c * h.Nn + node] += t[c] * jac * I[a];
      }
    SDME_CUDA(cudaMemcpyAsync(f_dev, f.data(), sizeof(double) * ctx->ndof, cudaMemcpyHostToDevice, ctx->stream));
    SDME_CUDA(cudaStreamSynchronize(ctx->stream));
    return SDME_OK;
  }
  // 1D integrals I_j = int_{-1}^{1} phi_j
  std::vector<double> I(n, 0.0);
  for (int q = 0; q < Q; ++q)
    for (int j = 0; j < n; ++j) I[j] += h.W[q] * h.B[q * n + j];
  const int axis = face / 2, side = face % 2;
  const int ta = (axis == 0) ? 1 : 0, tb = (axis == 2) ? 1 : 2;
  const double hl[3] = {ctx->mesh.length[0] / ctx->mesh.nelem[0], ctx->mesh.length[1] / ctx->mesh.nelem[1],
                        ctx->mesh.length[2] / ctx->mesh.nelem[2]};
  const double jac = 0.25 * hl[ta] * hl[tb];
  std::vector<double> f(ctx->ndof, 0.0);
  const int fixed = side ? h.N[axis] - 1 : 0;
  for (int ea = 0; ea < h.ne[ta]; ++ea)
    for (int eb = 0; eb < h.ne[tb]; ++eb)
      for (int a = 0; a < n; ++a)
        for (int bq = 0; bq < n; ++bq) {
          int idx[3];
          idx[axis] = fixed;
          idx[ta] = ea * P + a;
          idx[tb] = eb * P + bq;
          const int64_t node = ((int64_t)idx[2] * h.N[1] + idx[1]) * h.N[0] + idx[0];
          const double w = jac * I[a] * I[bq];
          for (int c = 0; c < 3; ++c) f[c * h.Nn + node] += t[c] * w;
        }
  SDME_CUDA(cudaMemcpyAsync(f_dev, f.data(), sizeof(double) * ctx->ndof, cudaMemcpyHostToDevice, ctx->stream));
  SDME_CUDA(cudaStreamSynchronize(ctx->stream));
  return SDME_OK;
}

sdme_status sdme_implicit_newmark_step(sdme_ctx* ctx, sdme_state* state, double dt, const double* P_next_dev,
                                       const sdme_newton_opts* opts, sdme_step_stats* stats) {
  if (!ctx || !state || !state->u || !state->v || !state->a || !P_next_dev || !(dt > 0.0)) return SDME_EINVAL;
  if (ctx->mlump) return SDME_EUNSUPPORTED;
  sdme_newton_opts o{0.25, 0.5, 1e-8, 30, 1e-10, 1e-4, 20000};
  if (opts) o = *opts;
  if (!(o.beta > 0.0) || o.max_newton < 0 || o.pcg_maxit < 1) return SDME_EINVAL;
  sdme_step_stats st{};
  const int64_t nd = ctx->ndof;
  const double b1 = 1.0 / (o.beta * dt * dt), b2 = 1.0 / (o.beta * dt), b3 = (1.0 - 2.0 * o.beta) / (2.0 * o.beta);
  cudaStream_t s = ctx->stream;
  SDME_CUDA(cudaMemcpyAsync(ctx->un, state->u, sizeof(double) * nd, cudaMemcpyDeviceToDevice, s));
  k_newmark_ahat<<<kVecBlocks, kVecThreads, 0, s>>>(nd, ctx->un, state->v, state->a, b1, b2, b3, ctx->ahat);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  SDME_TRY(sdme_mass_apply(ctx, ctx->ahat, ctx->mhat));
  const sdme_status result = newton_core(ctx, state->u, P_next_dev, b1, ctx->mhat, o, st);
  if (result != SDME_OK) {
    // the step did not converge: the state stays at t_n (u back to u_n)
    if (result != SDME_ECUDA) {
      SDME_CUDA(cudaMemcpyAsync(state->u, ctx->un, sizeof(double) * nd, cudaMemcpyDeviceToDevice, s));
      SDME_CUDA(cudaStreamSynchronize(s));
    }
    if (stats) *stats = st;
    return result;
  }
  k_newmark_final<<<kVecBlocks, kVecThreads, 0, s>>>(nd, state->u, ctx->ahat, b1, dt, o.gamma, state->v, state->a);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  SDME_CUDA(cudaStreamSynchronize(s));
  if (stats) *stats = st;
  return result;
}

sdme_status sdme_static_solve(sdme_ctx* ctx, double* u_dev, const double* P_dev, const sdme_newton_opts* opts,
                              sdme_step_stats* stats) {
  if (!ctx || !u_dev || !P_dev) return SDME_EINVAL;
  sdme_newton_opts o{0.25, 0.5, 1e-8, 50, 1e-12, 1e-4, 20000};
  if (opts) o = *opts;
  if (o.max_newton < 0 || o.pcg_maxit < 1) return SDME_EINVAL;
  sdme_step_stats st{};
  const sdme_status result = newton_core(ctx, u_dev, P_dev, 0.0, nullptr, o, st);
  if (result == SDME_ECUDA || result == SDME_NONPOSITIVE_J) return result;
  SDME_CUDA(cudaStreamSynchronize(ctx->stream));
  if (stats) *stats = st;
  return result;
}

sdme_status sdme_explicit_start(sdme_ctx* ctx, sdme_explicit_state* st, double dt, const double* P0_dev,
                                const double* v0_dev, double rtol, int maxit) {
  if (!ctx || !st || !st->u || !st->u_prev || !st->a || !P0_dev || !v0_dev || !(dt > 0.0) || maxit < 1)
    return SDME_EINVAL;
  SDME_TRY(residual_launch(ctx, 0.0, st->u, ctx->y, false));
  k_residual_combine<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, P0_dev, nullptr, ctx->y, ctx->psi,
                                                                  ctx->partial, ctx->dcount, ctx->dscal);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  SDME_TRY(sync_and_check(ctx));
  int its = 0;
  double rel = 0.0;
  sdme_status ps = mass_solve_core(ctx, ctx->psi, st->a, rtol, maxit, &its, &rel);
  if (ps != SDME_OK) return ps;
  k_cd_start<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, st->u, v0_dev, st->a, dt, st->u_prev);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  SDME_CUDA(cudaStreamSynchronize(ctx->stream));
  return SDME_OK;
}

sdme_status sdme_explicit_step(sdme_ctx* ctx, sdme_explicit_state* st, double dt, const double* Pn_dev, double rtol,
                               int maxit, int* pcg_iters) {
  if (!ctx || !st || !st->u || !st->u_prev || !st->a || !Pn_dev || !(dt > 0.0) || maxit < 1) return SDME_EINVAL;
  SDME_TRY(residual_launch(ctx, 0.0, st->u, ctx->y, false));
  if (ctx->mlump) {
    // diagonal mass: acceleration and update in one pass, no solve
    k_cd_lumped<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, st->u, Pn_dev, ctx->y, ctx->mlump, dt * dt,
                                                             st->a, st->u_prev);
    SDME_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
    if (pcg_iters) *pcg_iters = 0;
    double* t = st->u;
    st->u = st->u_prev;
    st->u_prev = t;
    return sync_and_check(ctx);
  }
  k_residual_combine<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, Pn_dev, nullptr, ctx->y, ctx->psi,
                                                                  ctx->partial, ctx->dcount, ctx->dscal);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  int its = 0;
  double rel = 0.0;
  sdme_status ps = pcg_dispatch(ctx, 1.0, ctx->psi, st->a, rtol, maxit, &its, &rel, true);
  if (pcg_iters) *pcg_iters = its;
  if (ps != SDME_OK) return ps;
  // u_{n+1} = 2 u_n - u_{n-1} + dt^2 a_n, written over u_{n-1}; then swap
  k_cd_update<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, st->u, st->a, dt * dt, st->u_prev);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  double* t = st->u;
  st->u = st->u_prev;
  st->u_prev = t;
  return sync_and_check(ctx);
}

sdme_status sdme_energy(sdme_ctx* ctx, const double* u_dev, const double* v_dev, double* kinetic, double* strain) {
  if (!ctx) return SDME_EINVAL;
  if (kinetic) {
    if (!v_dev) return SDME_EINVAL;
    SDME_TRY(sdme_mass_apply(ctx, v_dev, ctx->y));
    double vmv = 0.0;
    SDME_TRY(dot_host(ctx, v_dev, ctx->y, &vmv));
    *kinetic = 0.5 * vmv;
  }
  if (strain) {
    if (!u_dev) return SDME_EINVAL;
    SDME_CUDA(dispatch_P(ctx->h.P, [&](auto Pc) {
      return launch_energy<decltype(Pc)::value>(ctx->h, u_dev, ctx->partial, ctx->dcount, ctx->dscal, ctx->err,
                                                ctx->stream);
    }));
    ctx->kernel_launches += 1;
    SDME_CUDA(cudaMemcpyAsync(ctx->dscal_h, ctx->dscal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    SDME_TRY(sync_and_check(ctx));
    *strain = ctx->dscal_h[0];
  }
  return SDME_OK;
}

sdme_status sdme_estimate_dt_crit(sdme_ctx* ctx, const double* u_dev, int iters, double* dt_crit,
                                  double* lambda_max) {
  if (!ctx || !u_dev || iters < 1) return SDME_EINVAL;
  // linearise at u, then power iteration x <- M^{-1} K_T x / |.| with the
  // Rayleigh quotient x.Kx / x.Mx; constrained DOFs stay zero
  SDME_TRY(residual_launch(ctx, 0.0, u_dev, ctx->y));
  SDME_TRY(sync_and_check(ctx));
  double* x = ctx->du;
  double* Kx = ctx->ahat;
  double* Mx = ctx->mhat;
  k_fill_hash<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, x, 12345u);
  SDME_CUDA(cudaGetLastError());
  double lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    double xx = 0.0;
    SDME_TRY(dot_host(ctx, x, x, &xx));
    if (!(xx > 0.0)) return SDME_NAN;
    k_scale<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->ndof, 1.0 / std::sqrt(xx), x);
    k_mask_init<double><<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, x, Kx);
    SDME_CUDA(cudaGetLastError());
    SDME_TRY((tangent_launch<double, double>(ctx, 0.0, x, Kx, nullptr, nullptr)));
    SDME_TRY(sdme_mass_apply(ctx, x, Mx));
    double xKx = 0.0, xMx = 0.0;
    SDME_TRY(dot_host(ctx, x, Kx, &xKx));
    SDME_TRY(dot_host(ctx, x, Mx, &xMx));
    lam = xKx / xMx;
    int its = 0;
    double rel = 0.0;
    sdme_status ps = mass_solve_core(ctx, Kx, x, 1e-6, 2000, &its, &rel);
    if (ps != SDME_OK && ps != SDME_PCG_MAXIT) return ps;
    ctx->kernel_launches += 3;
  }
  if (!(lam > 0.0)) return SDME_NAN;
  if (lambda_max) *lambda_max = lam;
  if (dt_crit) *dt_crit = 2.0 / std::sqrt(lam);
  return SDME_OK;
}

sdme_status sdme_body_load(sdme_ctx* ctx, const double* fq_dev, double* f_dev) {
  if (ctx && ctx->h.dim != 3) return SDME_EUNSUPPORTED;
  if (!ctx || !fq_dev || !f_dev) return SDME_EINVAL;
  SDME_CUDA(cudaMemsetAsync(f_dev, 0, sizeof(double) * ctx->ndof, ctx->stream));
  SDME_CUDA(dispatch_P(ctx->h.P, [&](auto Pc) {
    return launch_body_load<decltype(Pc)::value>(ctx->h, fq_dev, f_dev, ctx->stream);
  }));
  ctx->kernel_launches += 1;
  return SDME_OK;
}

sdme_status sdme_mass_solve(sdme_ctx* ctx, const double* b_dev, double* x_dev, double rtol, int maxit, int* iters,
                            double* final_rel) {
  if (!ctx || !b_dev || !x_dev || maxit < 1 || !(rtol >= 0.0)) return SDME_EINVAL;
  return mass_solve_core(ctx, b_dev, x_dev, rtol, maxit, iters, final_rel);
}

sdme_status sdme_gauss_points(const sdme_ctx* ctx, double* xq, double* wq) {
  if (!ctx) return SDME_EINVAL;
  std::vector<double> x(ctx->Q), w(ctx->Q);
  gauss_legendre(ctx->Q, x.data(), w.data());
  for (int q = 0; q < ctx->Q; ++q) {
    if (xq) xq[q] = x[q];
    if (wq) wq[q] = w[q];
  }
  return SDME_OK;
}

sdme_status sdme_gauss_point_coords(sdme_ctx* ctx, double* X_dev) {
  if (!ctx || !X_dev) return SDME_EINVAL;
  if (ctx->h.dim != 3) return SDME_EUNSUPPORTED;
  GaussCoordParams p{};
  std::vector<double> x(ctx->Q), w(ctx->Q);
  gauss_legendre(ctx->Q, x.data(), w.data());
  for (int q = 0; q < ctx->Q; ++q) p.xq[q] = x[q];
  for (int d = 0; d < 3; ++d) {
    p.h[d] = ctx->mesh.length[d] / ctx->mesh.nelem[d];
    p.ne[d] = ctx->mesh.nelem[d];
  }
  p.Q = ctx->Q;
  const int64_t total = (int64_t)ctx->h.nelem * ctx->Q * ctx->Q * ctx->Q;
  k_gauss_coords<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(p, total, X_dev);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  return SDME_OK;
}

const char* sdme_cuda_error_string(const sdme_ctx* ctx) {
  if (!ctx) return "no context";
  return cudaGetErrorString(ctx->last_cuda != cudaSuccess ? ctx->last_cuda : ctx->last_timing_error);
}

sdme_status sdme_set_tangent_grid(sdme_ctx* ctx, int ctas) {
  if (!ctx || ctas < -1) return SDME_EINVAL;
  int grid = ctas;
  if (ctas == -1) {
    int per_sm = 0, dev = 0, sms = 0;
    SDME_CUDA(dispatch_P(ctx->h.P, [&](auto Pc) {
      constexpr int P = decltype(Pc)::value;
      per_sm = ctx->prec == SDME_MIXED_FP32 ? tangent_resident_ctas<P, float, float>()
                                             : tangent_resident_ctas<P, double, double>();
      return cudaSuccess;
    }));
    SDME_CUDA(cudaGetDevice(&dev));
    SDME_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return SDME_ECUDA;
    grid = per_sm * sms;
  }
  ctx->tan_grid = grid;
  if (ctx->gexec[0]) {  // the captured PCG chunk holds the old launch shape
    cudaGraphExecDestroy(ctx->gexec[0]);
    ctx->gexec[0] = nullptr;
  }
  return SDME_OK;
}

int sdme_get_tangent_grid(const sdme_ctx* ctx) { return ctx ? ctx->tan_grid : -1; }

sdme_status sdme_set_refinement(sdme_ctx* ctx, int max_restarts) {
  if (!ctx || max_restarts < 0) return SDME_EINVAL;
  ctx->refine_max = max_restarts;
  return SDME_OK;
}

sdme_status sdme_set_timing(sdme_ctx* ctx, int enable) {
  if (!ctx) return SDME_EINVAL;
  ctx->timing = enable != 0;
  return SDME_OK;
}

sdme_status sdme_get_timing(sdme_ctx* ctx, sdme_timing* out) {
  if (!ctx || !out) return SDME_EINVAL;
  out->tangent_ms = ctx->tangent_ms;
  out->tangent_launches = ctx->tangent_launches;
  out->kernel_launches = ctx->kernel_launches;
  return SDME_OK;
}

sdme_status sdme_tape_create(sdme_ctx* ctx, int nsteps, int every, sdme_tape** out) {
  if (!ctx || !out || nsteps < 1 || every < 1) return SDME_EINVAL;
  if (ctx->h.dim != 3) return SDME_EUNSUPPORTED;
  *out = nullptr;
  sdme_tape* tp = new (std::nothrow) sdme_tape();
  if (!tp) return SDME_ENOMEM;
  tp->ctx = ctx;
  tp->nsteps = nsteps;
  tp->every = std::min(every, nsteps);
  tp->nck = (nsteps + tp->every - 1) / tp->every;
  const size_t nd = (size_t)ctx->ndof;
  bool ok = dalloc(&tp->f, nd) == cudaSuccess && dalloc(&tp->ck, 2 * nd * tp->nck) == cudaSuccess &&
            dalloc(&tp->seg, nd * tp->every) == cudaSuccess;
  for (double*& p : tp->v) ok = ok && dalloc(&p, nd) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    sdme_tape_destroy(tp);
    return SDME_ENOMEM;
  }
  *out = tp;
  return SDME_OK;
}

sdme_status sdme_tape_destroy(sdme_tape* tp) {
  if (!tp) return SDME_OK;
  if (tp->ctx) cudaStreamSynchronize(tp->ctx->stream);
  for (double* p : {tp->f, tp->ck, tp->seg}) if (p) cudaFree(p);
  for (double* p : tp->v)
    if (p) cudaFree(p);
  delete tp;
  return SDME_OK;
}


sdme_status sdme_explicit_forward(sdme_ctx* ctx, sdme_tape* tp, double dt, const double* u0_dev, const double* v0_dev,
                                  const double* f_dev, const double* s_host, double rtol, int maxit, double* uN_dev) {
  if (!ctx || !tp || tp->ctx != ctx || !u0_dev || !v0_dev || !uN_dev || !(dt > 0.0) || maxit < 1 ||
      !(rtol >= 0.0) || (f_dev && !s_host))
    return SDME_EINVAL;
  tp->ran = false;
  tp->dt = dt;
  tp->rtol = rtol;
  tp->maxit = maxit;
  tp->have_f = f_dev != nullptr;
  tp->s.assign(tp->nsteps, 0.0);
  if (f_dev) {
    for (int n = 0; n < tp->nsteps; ++n) tp->s[n] = s_host[n];
    SDME_TRY(copy_vec(ctx, tp->f, f_dev));
  }
  const size_t nd = (size_t)ctx->ndof;
  sdme_explicit_state st{tp->v[0], tp->v[1], tp->v[2]};
  SDME_TRY(copy_vec(ctx, st.u, u0_dev));
  SDME_TRY(tape_load(tp, 0));
  SDME_TRY(sdme_explicit_start(ctx, &st, dt, tp->v[3], v0_dev, rtol, maxit));
  for (int n = 0; n < tp->nsteps; ++n) {
    if (n % tp->every == 0) {
      double* c = tp->ck + 2 * nd * (n / tp->every);
      SDME_TRY(copy_vec(ctx, c, st.u));
      SDME_TRY(copy_vec(ctx, c + nd, st.u_prev));
    }
    SDME_TRY(tape_load(tp, n));
    SDME_TRY(sdme_explicit_step(ctx, &st, dt, tp->v[3], rtol, maxit, nullptr));
  }
  SDME_TRY(copy_vec(ctx, uN_dev, st.u));
  SDME_CUDA(cudaStreamSynchronize(ctx->stream));
  tp->ran = true;
  return SDME_OK;
}

sdme_status sdme_explicit_adjoint(sdme_ctx* ctx, sdme_tape* tp, const double* gN_dev, double* gmu, double* glambda,
                                  double* gu0_dev, double* gv0_dev, double* gf_dev) {
  if (!ctx || !tp || tp->ctx != ctx || !gN_dev || !tp->ran) return SDME_EINVAL;
  const size_t nd = (size_t)ctx->ndof;
  const int N = tp->nsteps;
  const double dt = tp->dt, dt2 = dt * dt;
  double* g2 = tp->v[4];  // g_{n+2}
  double* g1 = tp->v[5];  // g_{n+1}
  SDME_CUDA(cudaMemsetAsync(g2, 0, sizeof(double) * nd, ctx->stream));
  SDME_TRY(copy_vec(ctx, g1, gN_dev));
  if (gf_dev) SDME_CUDA(cudaMemsetAsync(gf_dev, 0, sizeof(double) * nd, ctx->stream));
  double gth[2] = {0.0, 0.0};
  for (int k = tp->nck - 1; k >= 0; --k) {
    const int n0 = k * tp->every, n1 = std::min(n0 + tp->every, N);
    // recompute u_{n0} .. u_{n1-1} from the checkpoint (u_{n0}, u_{n0-1})
    sdme_explicit_state st{tp->v[0], tp->v[1], tp->v[2]};
    const double* c = tp->ck + 2 * nd * k;
    SDME_TRY(copy_vec(ctx, st.u, c));
    SDME_TRY(copy_vec(ctx, st.u_prev, c + nd));
    SDME_TRY(copy_vec(ctx, tp->seg, c));
    for (int n = n0; n < n1 - 1; ++n) {
      SDME_TRY(tape_load(tp, n));
      SDME_TRY(sdme_explicit_step(ctx, &st, dt, tp->v[3], tp->rtol, tp->maxit, nullptr));
      SDME_TRY(copy_vec(ctx, tp->seg + nd * (n + 1 - n0), st.u));
    }
    // reverse sweep over the segment: g_n from g_{n+1}, g_{n+2}
    for (int n = n1 - 1; n >= n0; --n) {
      SDME_TRY(adjoint_kernel_step(tp, tp->seg + nd * (n - n0), g1, dt2, tp->s[n], gth, gf_dev));
      k_adj_step<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, g1, g2, tp->v[7], dt2, g2);
      SDME_CUDA(cudaGetLastError());
      ctx->kernel_launches += 1;
      std::swap(g1, g2);  // g1 <- g_n, g2 <- g_{n+1}
    }
  }
  // start-up: g1 = g_0, g2 = g_1; rhs = g_{-1} = -g_1 on free DOFs
  double* rhs = tp->v[8];
  k_masked_scale<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, g2, -1.0, rhs);
  SDME_CUDA(cudaGetLastError());
  ctx->kernel_launches += 1;
  SDME_TRY(adjoint_kernel_step(tp, tp->ck, rhs, 0.5 * dt2, tp->s[0], gth, gf_dev));
  if (gu0_dev || gv0_dev) {
    k_adj_start<<<kVecBlocks, kVecThreads, 0, ctx->stream>>>(ctx->mi, g1, g2, tp->v[7], 0.5 * dt2, dt, gu0_dev,
                                                             gv0_dev);
    SDME_CUDA(cudaGetLastError());
    ctx->kernel_launches += 1;
  }
  SDME_CUDA(cudaStreamSynchronize(ctx->stream));
  if (gmu) *gmu = gth[0];
  if (glambda) *glambda = gth[1];
  return SDME_OK;
}

}  // extern "C"
