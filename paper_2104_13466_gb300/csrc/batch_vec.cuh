// Per-DOF kernels over a batch of independent meshes.  The vectors of all
// problems are concatenated (each problem's segment starts on a 64-byte
// boundary); every CTA belongs to one problem (cta_prob), walks that
// problem's segment with the problem's share of the grid, and per-problem
// reductions are finished by the last of the problem's CTAs to arrive
// (fixed summation order, no waiting).
#pragma once

#include "vec_kernels.cuh"

namespace sdme {

struct BatchVecInfo {
  MeshInfo mi;     // the problem's lattice (mi.ndof: its DOF count)
  int64_t off;     // offset of its segment in the concatenated vectors
  int cta0, ncta;  // its CTAs: [cta0, cta0 + ncta)
};

struct BatchCta {
  MeshInfo mi;
  int64_t off, t0, stride;
  int p, cta0, ncta;
  __device__ __forceinline__ BatchCta(const BatchVecInfo* __restrict__ info, const int* __restrict__ cta_prob) {
    p = cta_prob[blockIdx.x];
    const BatchVecInfo& f = info[p];
    mi = f.mi;
    off = f.off;
    cta0 = f.cta0;
    ncta = f.ncta;
    t0 = (int64_t)(blockIdx.x - cta0) * blockDim.x + threadIdx.x;
    stride = (int64_t)ncta * blockDim.x;
  }
};

// per-problem sum of the CTA partials partial[w * blockIdx + j]
__device__ __forceinline__ double batch_partial_sum(const double* partial, const BatchCta& b, int w, int j) {
  double s = 0.0;
  for (int i = threadIdx.x; i < b.ncta; i += blockDim.x) s += ((const volatile double*)partial)[w * (b.cta0 + i) + j];
  return block_sum(s);
}

template <typename TV>
__global__ void __launch_bounds__(kVecThreads) kb_mask_init(const BatchVecInfo* __restrict__ info,
                                                            const int* __restrict__ cta_prob,
                                                            const TV* __restrict__ x, TV* __restrict__ y) {
  const BatchCta b(info, cta_prob);
  for (int64_t g = b.t0; g < b.mi.ndof; g += b.stride) y[b.off + g] = dof_constrained(b.mi, g) ? x[b.off + g] : TV(0);
}

template <typename TV>
__global__ void __launch_bounds__(kVecThreads) kb_diag_finish(const BatchVecInfo* __restrict__ info,
                                                              const int* __restrict__ cta_prob, TV* __restrict__ d,
                                                              int inverse) {
  const BatchCta b(info, cta_prob);
  for (int64_t g = b.t0; g < b.mi.ndof; g += b.stride) {
    const TV v = dof_constrained(b.mi, g) ? TV(1) : d[b.off + g];
    d[b.off + g] = inverse ? TV(1) / v : v;
  }
}

// psi = P + mhat - y (0 on constrained DOFs); out[p] = ||psi_p||^2.
__global__ void __launch_bounds__(kVecThreads) kb_residual_combine(const BatchVecInfo* __restrict__ info,
                                                                   const int* __restrict__ cta_prob,
                                                                   const double* __restrict__ Pl,
                                                                   const double* __restrict__ mhat,
                                                                   const double* __restrict__ y,
                                                                   double* __restrict__ psi,
                                                                   double* __restrict__ partial,
                                                                   unsigned int* counters, double* out) {
  const BatchCta b(info, cta_prob);
  double s = 0.0;
  for (int64_t g = b.t0; g < b.mi.ndof; g += b.stride) {
    const int64_t i = b.off + g;
    double v = 0.0;
    if (!dof_constrained(b.mi, g)) v = Pl[i] + mhat[i] - y[i];
    psi[i] = v;
    s += v * v;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  if (last_arrival(&counters[b.p], b.ncta)) {
    const double t = batch_partial_sum(partial, b, 1, 0);
    if (threadIdx.x == 0) {
      out[b.p] = t;
      counters[b.p] = 0;
    }
  }
}

// out[p] = ||x_p||^2 over all of the problem's DOFs
__global__ void __launch_bounds__(kVecThreads) kb_norm2(const BatchVecInfo* __restrict__ info,
                                                        const int* __restrict__ cta_prob,
                                                        const double* __restrict__ x, double* __restrict__ partial,
                                                        unsigned int* counters, double* out) {
  const BatchCta b(info, cta_prob);
  double s = 0.0;
  for (int64_t g = b.t0; g < b.mi.ndof; g += b.stride) {
    const double v = x[b.off + g];
    s += v * v;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  if (last_arrival(&counters[b.p], b.ncta)) {
    const double t = batch_partial_sum(partial, b, 1, 0);
    if (threadIdx.x == 0) {
      out[b.p] = t;
      counters[b.p] = 0;
    }
  }
}

// Jacobi-PCG initialisation per problem (as k_pcg_init); problems with
// active[p] == 0 start from a zero right-hand side, i.e. converge at once
// with x = 0.
template <typename TV>
__global__ void __launch_bounds__(kVecThreads) kb_pcg_init(const BatchVecInfo* __restrict__ info,
                                                           const int* __restrict__ cta_prob,
                                                           const double* __restrict__ rhs,
                                                           const TV* __restrict__ dinv, TV* __restrict__ x,
                                                           TV* __restrict__ r, TV* __restrict__ p, TV* __restrict__ q,
                                                           PcgScalars* scal, double* __restrict__ partial,
                                                           const int* __restrict__ active, double rtol, int maxit) {
  const BatchCta b(info, cta_prob);
  const bool act = active[b.p] != 0;
  double srz = 0.0, srr = 0.0;
  for (int64_t g = b.t0; g < b.mi.ndof; g += b.stride) {
    const int64_t i = b.off + g;
    const TV rv = (!act || dof_constrained(b.mi, g)) ? TV(0) : (TV)rhs[i];
    const TV z = dinv[i] * rv;
    r[i] = rv;
    p[i] = z;
    x[i] = TV(0);
    q[i] = TV(0);
    srz += (double)(rv * z);
    srr += (double)(rv * rv);
  }
  double a = srz, c = srr;
  block_sum2(a, c);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = c;
  }
  PcgScalars* sc = scal + b.p;
  if (last_arrival(&sc->counter2, b.ncta)) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < b.ncta; i += blockDim.x) {
      s0 += ((volatile double*)partial)[2 * (b.cta0 + i)];
      s1 += ((volatile double*)partial)[2 * (b.cta0 + i) + 1];
    }
    block_sum2(s0, s1);
    if (threadIdx.x == 0) {
      sc->rz = s0;
      sc->bb = s1;
      sc->rr = s1;
      sc->tol2 = rtol * rtol * s1;
      sc->iter = 0;
      sc->maxit = maxit;
      sc->alpha = 0.0;
      sc->beta = 0.0;
      sc->pq = 0.0;
      sc->status = (s1 == 0.0) ? kPcgConverged : (isfinite(s1) ? kPcgRunning : kPcgBreakdown);
      sc->counter = 0;
      sc->counter2 = 0;
    }
  }
}

template <typename TV>
__global__ void __launch_bounds__(kVecThreads) kb_pcg_update(const BatchVecInfo* __restrict__ info,
                                                             const int* __restrict__ cta_prob, TV* __restrict__ x,
                                                             TV* __restrict__ r, const TV* __restrict__ p,
                                                             TV* __restrict__ q, const TV* __restrict__ dinv,
                                                             PcgScalars* scal, double* __restrict__ partial,
                                                             int* __restrict__ queue = nullptr) {
  // the persistent operator's work counter (if any) is free again: this
  // launch follows the operator, the next operator follows the direction
  if (queue && blockIdx.x == 0 && threadIdx.x == 0) *queue = 0;
  const BatchCta b(info, cta_prob);
  PcgScalars* sc = scal + b.p;
  if (sc->status != kPcgRunning) return;
  using V = typename Vec16<TV>::type;
  constexpr int W = Vec16<TV>::width;
  const TV alpha = (TV)sc->alpha;
  typename AccOf<TV>::type srz, srr;
  TV *xs = x + b.off, *rs = r + b.off, *qs = q + b.off;
  const TV *ps = p + b.off, *ds = dinv + b.off;
  const int64_t n = b.mi.ndof, nv = n / W;
  for (int64_t g = b.t0; g < nv; g += b.stride) {
    V xv = reinterpret_cast<const V*>(xs)[g];
    V rv = reinterpret_cast<const V*>(rs)[g];
    V pv = reinterpret_cast<const V*>(ps)[g];
    V qv = reinterpret_cast<const V*>(qs)[g];
    V dv = reinterpret_cast<const V*>(ds)[g];
    TV vrz = TV(0), vrr = TV(0);
#pragma unroll
    for (int i = 0; i < W; ++i) {
      lane(xv, i) += alpha * lane(pv, i);
      const TV ri = lane(rv, i) - alpha * lane(qv, i);
      lane(rv, i) = ri;
      vrz += ri * (lane(dv, i) * ri);
      vrr += ri * ri;
    }
    srz.add(vrz);
    srr.add(vrr);
    reinterpret_cast<V*>(xs)[g] = xv;
    reinterpret_cast<V*>(rs)[g] = rv;
    reinterpret_cast<V*>(qs)[g] = V{};
  }
  for (int64_t g = nv * W + b.t0; g < n; g += b.stride) {
    const TV qv = qs[g];
    xs[g] += alpha * ps[g];
    const TV rv = rs[g] - alpha * qv;
    rs[g] = rv;
    qs[g] = TV(0);
    srz.add(rv * (ds[g] * rv));
    srr.add(rv * rv);
  }
  double a = srz.value(), c = srr.value();
  block_sum2(a, c);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = c;
  }
  if (last_arrival(&sc->counter2, b.ncta)) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < b.ncta; i += blockDim.x) {
      s0 += ((volatile double*)partial)[2 * (b.cta0 + i)];
      s1 += ((volatile double*)partial)[2 * (b.cta0 + i) + 1];
    }
    block_sum2(s0, s1);
    if (threadIdx.x == 0) {
      sc->iter += 1;
      sc->rr = s1;
      sc->beta = s0 / sc->rz;
      sc->rz = s0;
      if (!isfinite(s1) || !isfinite(s0)) sc->status = kPcgBreakdown;
      else if (s1 <= sc->tol2) sc->status = kPcgConverged;
      else if (sc->iter >= sc->maxit) sc->status = kPcgMaxit;
      sc->counter2 = 0;
    }
  }
}

template <typename TV>
__global__ void __launch_bounds__(kVecThreads) kb_pcg_direction(const BatchVecInfo* __restrict__ info,
                                                                const int* __restrict__ cta_prob,
                                                                const TV* __restrict__ r, const TV* __restrict__ dinv,
                                                                TV* __restrict__ p, const PcgScalars* scal) {
  const BatchCta b(info, cta_prob);
  const PcgScalars* sc = scal + b.p;
  if (sc->status != kPcgRunning) return;
  using V = typename Vec16<TV>::type;
  constexpr int W = Vec16<TV>::width;
  const TV beta = (TV)sc->beta;
  const TV *rs = r + b.off, *ds = dinv + b.off;
  TV* ps = p + b.off;
  const int64_t n = b.mi.ndof, nv = n / W;
  for (int64_t g = b.t0; g < nv; g += b.stride) {
    V rv = reinterpret_cast<const V*>(rs)[g];
    V dv = reinterpret_cast<const V*>(ds)[g];
    V pv = reinterpret_cast<const V*>(ps)[g];
#pragma unroll
    for (int i = 0; i < W; ++i) lane(pv, i) = lane(dv, i) * lane(rv, i) + beta * lane(pv, i);
    reinterpret_cast<V*>(ps)[g] = pv;
  }
  for (int64_t g = nv * W + b.t0; g < n; g += b.stride) ps[g] = ds[g] * rs[g] + beta * ps[g];
}

}  // namespace sdme
