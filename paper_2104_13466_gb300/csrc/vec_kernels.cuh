// Per-DOF kernels: Dirichlet handling, Newton residual assembly, Newmark
// updates and the fused Jacobi-PCG vector steps.  Grid-stride loops over a
// fixed grid (a multiple of the SM count); float64 reductions finished by the
// last CTA to arrive (deterministic order, no waiting).
#pragma once

#include <type_traits>

#include "common.cuh"

namespace sdme {

constexpr int kVecThreads = 256;

// y = x on constrained DOFs, 0 elsewhere (start of a masked operator apply).
template <typename TV>
__global__ void __launch_bounds__(kVecThreads) k_mask_init(MeshInfo mi, const TV* __restrict__ x,
                                                           TV* __restrict__ y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x)
    y[g] = dof_constrained(mi, g) ? x[g] : TV(0);
}

// Diagonal post-processing: constrained -> 1; out = inverse ? 1/d : d.
template <typename TV>
__global__ void __launch_bounds__(kVecThreads) k_diag_finish(MeshInfo mi, TV* __restrict__ d, int inverse) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x) {
    TV v = dof_constrained(mi, g) ? TV(1) : d[g];
    d[g] = inverse ? TV(1) / v : v;
  }
}

// psi = P + mhat - y (mhat may be null), 0 on constrained DOFs; out = ||psi||^2.
static __global__ void __launch_bounds__(kVecThreads) k_residual_combine(MeshInfo mi, const double* __restrict__ Pl,
                                                                  const double* __restrict__ mhat,
                                                                  const double* __restrict__ y,
                                                                  double* __restrict__ psi,
                                                                  double* __restrict__ partial,
                                                                  unsigned int* counter, double* out) {
  double s = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (!dof_constrained(mi, g)) {
      v = (Pl ? Pl[g] : 0.0) - y[g];
      if (mhat) v += mhat[g];
    }
    psi[g] = v;
    s += v * v;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  if (last_block_done(counter)) {
    const double t = ordered_sum(partial, gridDim.x);
    if (threadIdx.x == 0) {
      *out = t;
      *counter = 0;
    }
  }
}

// out = ||x||^2 (all DOFs)
static __global__ void __launch_bounds__(kVecThreads) k_norm2(int64_t n, const double* __restrict__ x,
                                                       double* __restrict__ partial, unsigned int* counter,
                                                       double* out) {
  double s = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    s += x[g] * x[g];
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  if (last_block_done(counter)) {
    const double t = ordered_sum(partial, gridDim.x);
    if (threadIdx.x == 0) {
      *out = t;
      *counter = 0;
    }
  }
}

// ahat = b2 v + b3 a + b1 u_n, so that a(u) = b1 u - ahat (Newmark, Sec. 4.2)
static __global__ void __launch_bounds__(kVecThreads) k_newmark_ahat(int64_t n, const double* __restrict__ un,
                                                              const double* __restrict__ v,
                                                              const double* __restrict__ a, double b1, double b2,
                                                              double b3, double* __restrict__ ahat) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    ahat[g] = b2 * v[g] + b3 * a[g] + b1 * un[g];
}

// a_{n+1} = b1 u - ahat ; v_{n+1} = v_n + dt ((1 - gamma) a_n + gamma a_{n+1})
static __global__ void __launch_bounds__(kVecThreads) k_newmark_final(int64_t n, const double* __restrict__ u,
                                                               const double* __restrict__ ahat, double b1,
                                                               double dt, double gamma, double* __restrict__ v,
                                                               double* __restrict__ a) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const double an = a[g];
    const double a1 = b1 * u[g] - ahat[g];
    v[g] = v[g] + dt * ((1.0 - gamma) * an + gamma * a1);
    a[g] = a1;
  }
}

// y += alpha x, x given in TV (converted to float64)
template <typename TV>
__global__ void __launch_bounds__(kVecThreads) k_axpy(int64_t n, double alpha, const TV* __restrict__ x,
                                                      double* __restrict__ y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    y[g] += alpha * (double)x[g];
}

//----------------------------------------------------------------------------
// Jacobi PCG (CGD).  Vectors r, p, q, dinv in TV (dinv = 1 / diag).  The
// solution x is float64 (TV = double) or, with float32 vectors, either a
// float32 pair (hi, lo) holding hi + lo to about 48 bits (xl given), or a
// single float32 x (xl null) that the refined solves fold into a float64
// solution at every refinement check, so that it only ever holds one
// sweep's correction: a float32 x holding the whole solution would bound the
// float64 residual b - A x at about eps32 |A| |x|, and float64 arithmetic
// runs at a small fraction of the float32 rate on GB300.
//   init:      r = scale*b (0 on constrained), x = 0, q = 0, p = z = dinv r,
//              rz = r.z, bb = r.r
//   per iteration:  tangent kernel: q = A p, pq = p.q, alpha = rz / pq
//                   update:    r -= alpha q, q = 0,
//                              rz' = r.(dinv r), rr = r.r, test, beta = rz'/rz
//                   direction: x += alpha p (with the p the operator saw),
//                              p = dinv r + beta p
//   final:     after the iteration that meets the test (the direction kernel
//              then returns at once) the host issues x += alpha p.
//   restart:   r = a given float64 residual, p = z = dinv r (x, bb, tol2 and
//              the iteration count kept): the refinement step of the float32
//              solve.
// Dot products: each product in TV (float32 products of float32 vectors are
// summed four at a time, one 16-byte vector), accumulated per thread (float64,
// or for float32 vectors in the update a compensated float32 sum of about 48
// bits, FFSum) and reduced across threads in float64.
//----------------------------------------------------------------------------
template <typename TV>
__global__ void __launch_bounds__(kVecThreads) k_pcg_init(MeshInfo mi, const double* __restrict__ b, double scale,
                                                          const TV* __restrict__ dinv, TV* __restrict__ xh,
                                                          TV* __restrict__ xl, TV* __restrict__ r,
                                                          TV* __restrict__ p, TV* __restrict__ q, PcgScalars* scal,
                                                          double* __restrict__ partial, double rtol, int maxit) {
  double srz = 0.0, srr = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x) {
    const TV rv = dof_constrained(mi, g) ? TV(0) : (TV)(scale * b[g]);
    const TV z = dinv[g] * rv;
    r[g] = rv;
    p[g] = z;
    xh[g] = TV(0);
    if (xl) xl[g] = TV(0);
    q[g] = TV(0);
    srz += (double)(rv * z);
    srr += (double)(rv * rv);
  }
  double a = srz, c = srr;
  block_sum2(a, c);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = c;
  }
  if (last_block_done(&scal->counter2)) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
      s0 += ((volatile double*)partial)[2 * i];
      s1 += ((volatile double*)partial)[2 * i + 1];
    }
    block_sum2(s0, s1);
    if (threadIdx.x == 0) {
      scal->rz = s0;
      scal->bb = s1;
      scal->rr = s1;
      scal->tol2 = rtol * rtol * s1;
      scal->iter = 0;
      scal->maxit = maxit;
      scal->alpha = 0.0;
      scal->beta = 0.0;
      scal->pq = 0.0;
      scal->status = (s1 == 0.0) ? kPcgConverged : (isfinite(s1) ? kPcgRunning : kPcgBreakdown);
      scal->counter = 0;
      scal->counter2 = 0;
    }
  }
}

// 16-byte vector of TV used by the streaming PCG kernels.
template <typename TV>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int width = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int width = 2;
};

// 16-byte load cached in L2 only (no stale L1 line of a vector rewritten by
// an earlier launch)
__device__ __forceinline__ float4 ldcg_vec(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldcg_vec(const double2* p) { return __ldcg(p); }

// L2 evict-last access policy and 16-byte loads / stores under it (float32
// vectors; the float64 overloads are plain accesses): vectors that the next
// kernel reads again stay in L2 ahead of streamed data.
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float4 ld_el(const float4* p, uint64_t pol) {
  float4 v;
  asm("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_el(const double2* p, uint64_t) { return *p; }
__device__ __forceinline__ void st_el(float4* p, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_el(double2* p, double2 v, uint64_t) { *p = v; }

template <typename V>
__device__ __forceinline__ auto& lane(V& v, int i) {
  return reinterpret_cast<typename std::remove_reference<decltype(v.x)>::type*>(&v)[i];
}

// (hi, lo) += a * v for a float32 pair: the product split exactly by an FMA
// (Dekker / Ogita-Rump-Oishi TwoProduct), its high part added by Knuth's
// TwoSum, the low parts folded in and the pair renormalised.  The _rn
// intrinsics keep the compiler from fusing or reassociating the steps.
__device__ __forceinline__ void pair_axpy(float& hi, float& lo, float a, float v) {
  const float ph = __fmul_rn(a, v);
  const float pl = __fmaf_rn(a, v, -ph);
  const float s = __fadd_rn(hi, ph);
  const float bv = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(ph, bv));
  const float t = __fadd_rn(e, __fadd_rn(lo, pl));
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// x += alpha p (alpha from the scalars): the solution update of the
// iteration whose direction kernel returned at once (the test was met).
template <typename TV>
__global__ void __launch_bounds__(kVecThreads) k_pcg_xfinal(int64_t n, const TV* __restrict__ p,
                                                            TV* __restrict__ xh, TV* __restrict__ xl,
                                                            const PcgScalars* scal) {
  const double alpha = scal->alpha;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(TV) == 4) {
      if (xl) {
        float h = xh[g], l = xl[g];
        pair_axpy(h, l, (float)alpha, p[g]);
        xh[g] = h;
        xl[g] = l;
      } else {
        xh[g] += (float)alpha * p[g];
      }
    } else {
      xh[g] += alpha * p[g];
    }
  }
}

// out = hi + lo in float64 (TV = float), or a copy of x (TV = double).
// Refinement check of a single-x solve: x64 (+)= x in float64 (first: x64 =
// x), then x = 0 for the next sweep's correction.
template <typename TV>
__global__ void __launch_bounds__(kVecThreads) k_pcg_xfold(int64_t n, TV* __restrict__ xh, double* __restrict__ x64,
                                                           int first) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    x64[g] = (first ? 0.0 : x64[g]) + (double)xh[g];
    xh[g] = TV(0);
  }
}

// out = x64 + x in float64 (a single-x solve that folded at least once).
template <typename TV>
__global__ void __launch_bounds__(kVecThreads) k_pcg_xout64(int64_t n, const TV* __restrict__ xh,
                                                            const double* __restrict__ x64, double* __restrict__ out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    out[g] = x64[g] + (double)xh[g];
}

template <typename TV>
__global__ void __launch_bounds__(kVecThreads) k_pcg_xout(int64_t n, const TV* __restrict__ xh,
                                                          const TV* __restrict__ xl, double* __restrict__ out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    out[g] = xl ? (double)xh[g] + (double)xl[g] : (double)xh[g];
}

// Block size of the PCG update: 1024 threads, so that the CTAs that each
// sum the operator's per-element partials (the step length) are few.
constexpr int kUpdThreads = 1024;

template <typename TV>
__global__ void __launch_bounds__(kUpdThreads) k_pcg_update(int64_t n, TV* __restrict__ r, TV* __restrict__ q,
                                                            const TV* __restrict__ dinv, PcgScalars* scal,
                                                            double* __restrict__ partial,
                                                            const double* __restrict__ dot_partial = nullptr,
                                                            int nparts = 0) {
  using V = typename Vec16<TV>::type;
  constexpr int W = Vec16<TV>::width;
  const int64_t nv = n / W;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // the first chunk's loads do not depend on the step length: issue them
  // before it is summed so that their latency overlaps the sum.  r and 1/d
  // are not written by the operator launch this one may overlap (launched
  // as its programmatic dependent): they are read before pdl_wait(), through
  // L2; q after it
  V r0, q0, d0;
  const bool first = t0 < nv;
  if (first) {
    r0 = ldcg_vec(reinterpret_cast<const V*>(r) + t0);
    d0 = ldcg_vec(reinterpret_cast<const V*>(dinv) + t0);
  }
  pdl_wait();
  if (scal->status != kPcgRunning) return;
  pdl_trigger();
  if (first) q0 = reinterpret_cast<const V*>(q)[t0];
  double alpha_d;
  if (dot_partial) {
    // p . (A p) from the operator's per-element partials (which must not
    // alias `partial`), summed by every CTA in the same fixed order so that
    // all CTAs hold the same step length; CTA 0 publishes it
    // (one thread divides: a float64 division per thread of a 1024-thread
    // CTA would hold the float64 pipe for microseconds)
    const double pq = ordered_sum_prev(dot_partial, nparts);
    __shared__ double s_alpha;
    if (threadIdx.x == 0) {
      const double al = scal->rz / pq;
      s_alpha = (!(pq > 0.0) || !isfinite(al)) ? -1.0 : al;
      if (blockIdx.x == 0) {
        scal->pq = pq;
        scal->alpha = al;
        if (s_alpha < 0.0) scal->status = kPcgBreakdown;
      }
    }
    __syncthreads();
    alpha_d = s_alpha;
    if (alpha_d < 0.0) return;  // every CTA takes the same branch; none reaches the counter
  } else {
    alpha_d = scal->alpha;
  }
  const TV alpha = (TV)alpha_d;
  typename AccOf<TV>::type srz, srr;
  const uint64_t pol = l2_evict_last();   // r and 1/d kept in L2 for the direction update
  auto body = [&](V& rv, V& qv, V& dv, int64_t g) {
    TV vrz = TV(0), vrr = TV(0);
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const TV ri = lane(rv, i) - alpha * lane(qv, i);
      lane(rv, i) = ri;
      vrz += ri * (lane(dv, i) * ri);
      vrr += ri * ri;
    }
    srz.add(vrz);
    srr.add(vrr);
    st_el(reinterpret_cast<V*>(r) + g, rv, pol);
    reinterpret_cast<V*>(q)[g] = V{};
  };
  int64_t g = t0;
  if (first) {
    body(r0, q0, d0, t0);
    g += stride;
  }
  // two chunks per trip (six 16-byte loads in flight per thread), same chunk
  // order as a one-chunk loop
  for (; g + stride < nv; g += 2 * stride) {
    V rv[2], qv[2], dv[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      rv[u] = reinterpret_cast<const V*>(r)[g + u * stride];
      qv[u] = reinterpret_cast<const V*>(q)[g + u * stride];
      dv[u] = ld_el(reinterpret_cast<const V*>(dinv) + g + u * stride, pol);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) body(rv[u], qv[u], dv[u], g + u * stride);
  }
  for (; g < nv; g += stride) {
    V rv = reinterpret_cast<const V*>(r)[g];
    V qv = reinterpret_cast<const V*>(q)[g];
    V dv = ld_el(reinterpret_cast<const V*>(dinv) + g, pol);
    body(rv, qv, dv, g);
  }
  for (int64_t g = nv * W + t0; g < n; g += stride) {  // tail
    const TV qv = q[g];
    const TV rv = r[g] - alpha * qv;
    r[g] = rv;
    q[g] = TV(0);
    srz.add(rv * (dinv[g] * rv));
    srr.add(rv * rv);
  }
  double a, c;
  if constexpr (sizeof(TV) == 4) {
    block_sum2_ff(srz, srr, a, c);
  } else {
    a = srz.value();
    c = srr.value();
    block_sum2(a, c);
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = c;
  }
  if (last_block_done(&scal->counter2)) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
      s0 += ((volatile double*)partial)[2 * i];
      s1 += ((volatile double*)partial)[2 * i + 1];
    }
    block_sum2(s0, s1);
    if (threadIdx.x == 0) {
      scal->iter += 1;
      scal->rr = s1;
      scal->beta = s0 / scal->rz;
      scal->rz = s0;
      if (!isfinite(s1) || !isfinite(s0)) scal->status = kPcgBreakdown;
      else if (s1 <= scal->tol2) scal->status = kPcgConverged;
      else if (scal->iter >= scal->maxit) scal->status = kPcgMaxit;
      scal->counter2 = 0;
    }
  }
}

template <typename TV>
__global__ void __launch_bounds__(kVecThreads) k_pcg_direction(int64_t n, const TV* __restrict__ r,
                                                               const TV* __restrict__ dinv, TV* __restrict__ p,
                                                               TV* __restrict__ xh, TV* __restrict__ xl,
                                                               const PcgScalars* scal) {
  using V = typename Vec16<TV>::type;
  constexpr int W = Vec16<TV>::width;
  const int64_t nv = n / W;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // p, x and 1/d of the first chunk are not written by the update this
  // launch may overlap (as its programmatic dependent): read them before
  // pdl_wait(), through L2; r, the scalars and the status after it
  V p0, h0, d0;
  const bool first = t0 < nv;
  if (first) {
    p0 = ldcg_vec(reinterpret_cast<const V*>(p) + t0);
    h0 = ldcg_vec(reinterpret_cast<const V*>(xh) + t0);
    d0 = ldcg_vec(reinterpret_cast<const V*>(dinv) + t0);
  }
  pdl_wait();
  if (scal->status != kPcgRunning) return;
  pdl_trigger();
  const TV beta = (TV)scal->beta;
  const double alpha_d = scal->alpha;
  const TV alpha = (TV)alpha_d;
  for (int64_t g = t0; g < nv; g += stride) {
    V rv = reinterpret_cast<const V*>(r)[g];
    V dv, pv, hv;
    if (g == t0) {
      dv = d0;
      pv = p0;
      hv = h0;
    } else {
      dv = reinterpret_cast<const V*>(dinv)[g];
      pv = reinterpret_cast<const V*>(p)[g];
      hv = reinterpret_cast<const V*>(xh)[g];
    }
    if constexpr (sizeof(TV) == 4) {
      if (xl) {
        V lv = reinterpret_cast<const V*>(xl)[g];
#pragma unroll
        for (int i = 0; i < W; ++i) pair_axpy(lane(hv, i), lane(lv, i), alpha, lane(pv, i));
        reinterpret_cast<V*>(xl)[g] = lv;
      } else {
#pragma unroll
        for (int i = 0; i < W; ++i) lane(hv, i) += alpha * lane(pv, i);
      }
    } else {
#pragma unroll
      for (int i = 0; i < W; ++i) lane(hv, i) += alpha * lane(pv, i);
    }
    reinterpret_cast<V*>(xh)[g] = hv;
#pragma unroll
    for (int i = 0; i < W; ++i) lane(pv, i) = lane(dv, i) * lane(rv, i) + beta * lane(pv, i);
    reinterpret_cast<V*>(p)[g] = pv;
  }
  for (int64_t g = nv * W + t0; g < n; g += stride) {
    const TV pg = p[g];
    if constexpr (sizeof(TV) == 4) {
      if (xl) {
        float h = xh[g], l = xl[g];
        pair_axpy(h, l, alpha, pg);
        xh[g] = h;
        xl[g] = l;
      } else {
        xh[g] += alpha * pg;
      }
    } else {
      xh[g] += alpha * pg;
    }
    p[g] = dinv[g] * r[g] + beta * pg;
  }
}

template <typename TV>
__global__ void __launch_bounds__(kVecThreads) k_pcg_restart(MeshInfo mi, const double* __restrict__ rt,
                                                             const TV* __restrict__ dinv, TV* __restrict__ r,
                                                             TV* __restrict__ p, TV* __restrict__ q, PcgScalars* scal,
                                                             double* __restrict__ partial) {
  double srz = 0.0, srr = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x) {
    const TV rv = dof_constrained(mi, g) ? TV(0) : (TV)rt[g];
    const TV z = dinv[g] * rv;
    r[g] = rv;
    p[g] = z;
    q[g] = TV(0);
    srz += (double)(rv * z);
    srr += (double)(rv * rv);
  }
  double a = srz, c = srr;
  block_sum2(a, c);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = c;
  }
  if (last_block_done(&scal->counter2)) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
      s0 += ((volatile double*)partial)[2 * i];
      s1 += ((volatile double*)partial)[2 * i + 1];
    }
    block_sum2(s0, s1);
    if (threadIdx.x == 0) {
      scal->rz = s0;
      scal->rr = s1;
      scal->alpha = 0.0;
      scal->beta = 0.0;
      scal->pq = 0.0;
      if (!isfinite(s0) || !isfinite(s1)) scal->status = kPcgBreakdown;
      else if (s1 <= scal->tol2) scal->status = kPcgConverged;
      else if (scal->iter >= scal->maxit) scal->status = kPcgMaxit;
      else scal->status = kPcgRunning;
      scal->counter = 0;
      scal->counter2 = 0;
    }
  }
}

// out = scale * x (TV -> float64)
template <typename TV>
__global__ void __launch_bounds__(kVecThreads) k_to_double(int64_t n, const TV* __restrict__ x, double scale,
                                                           double* __restrict__ out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    out[g] = scale * (double)x[g];
}

// Central-difference start-up (Sec. 4.1): u_prev = u0 - dt v0 + dt^2/2 a0 on
// free DOFs, u0 on constrained ones.
static __global__ void __launch_bounds__(kVecThreads) k_cd_start(MeshInfo mi, const double* __restrict__ u,
                                                          const double* __restrict__ v, const double* __restrict__ a,
                                                          double dt, double* __restrict__ u_prev) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x)
    u_prev[g] = dof_constrained(mi, g) ? u[g] : u[g] - dt * v[g] + 0.5 * dt * dt * a[g];
}

// Central-difference update (eq. Motion_explicit2): out (holding u_{n-1})
// <- 2 u_n - u_{n-1} + dt^2 a_n on free DOFs, u_n on constrained ones.
static __global__ void __launch_bounds__(kVecThreads) k_cd_update(MeshInfo mi, const double* __restrict__ u,
                                                           const double* __restrict__ a, double dt2,
                                                           double* __restrict__ u_prev) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x) {
    const double un = u[g];
    u_prev[g] = dof_constrained(mi, g) ? un : 2.0 * un - u_prev[g] + dt2 * a[g];
  }
}

// out = x . y (float64, fixed-order finalize by the last CTA)
static __global__ void __launch_bounds__(kVecThreads) k_dot(int64_t n, const double* __restrict__ x,
                                                     const double* __restrict__ y, double* __restrict__ partial,
                                                     unsigned int* counter, double* out) {
  double s = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    s += x[g] * y[g];
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  if (last_block_done(counter)) {
    const double t = ordered_sum(partial, gridDim.x);
    if (threadIdx.x == 0) {
      *out = t;
      *counter = 0;
    }
  }
}

// Deterministic pseudo-random start vector in [-1, 1] (integer hash of the
// index), zero on constrained DOFs.
static __global__ void __launch_bounds__(kVecThreads) k_fill_hash(MeshInfo mi, double* __restrict__ x, unsigned seed) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)g * 2654435761u ^ seed;
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    h *= 0x846ca68bu;
    h ^= h >> 16;
    x[g] = dof_constrained(mi, g) ? 0.0 : (double)h * (2.0 / 4294967295.0) - 1.0;
  }
}

static __global__ void __launch_bounds__(kVecThreads) k_scale(int64_t n, double s, double* __restrict__ x) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    x[g] *= s;
}


// Discrete adjoint of one central-difference step.  The step maps
// (u_n, u_{n-1}) to u_{n+1} = 2 u_n - u_{n-1} + dt^2 A (P_n - R(u_n)) on free
// DOFs and u_n on constrained ones (A: mass inverse on the free DOFs), so
// g_n = dJ/du_n = [2 g_{n+1} - g_{n+2} | g_{n+1}] - dt^2 K_T(u_n) z_n with
// z_n = A g_{n+1}.  out may alias g2 (element-wise in place).
static __global__ void __launch_bounds__(kVecThreads) k_adj_step(MeshInfo mi, const double* g1, const double* g2,
                                                          const double* __restrict__ Kz, double dt2, double* out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x) {
    const double a = g1[g];
    const double b = dof_constrained(mi, g) ? a : 2.0 * a - g2[g];
    out[g] = b - dt2 * Kz[g];
  }
}

// out = a x on free DOFs, 0 on constrained ones.
static __global__ void __launch_bounds__(kVecThreads) k_masked_scale(MeshInfo mi, const double* __restrict__ x, double a,
                                                              double* __restrict__ out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x)
    out[g] = dof_constrained(mi, g) ? 0.0 : a * x[g];
}

// Adjoint of the start-up u_{-1} = u_0 - dt v_0 + dt^2/2 A (P_0 - R(u_0)) (free
// DOFs): with g_{-1} = -g_1 on free DOFs and z = A g_{-1},
// dJ/du_0 = g_0 + g_{-1} - dt^2/2 K_T(u_0) z and dJ/dv_0 = -dt g_{-1}.
static __global__ void __launch_bounds__(kVecThreads) k_adj_start(MeshInfo mi, const double* __restrict__ g0,
                                                           const double* __restrict__ g1,
                                                           const double* __restrict__ Kz, double half_dt2, double dt,
                                                           double* __restrict__ gu0, double* __restrict__ gv0) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x) {
    const double gm1 = dof_constrained(mi, g) ? 0.0 : -g1[g];
    if (gu0) gu0[g] = g0[g] + gm1 - half_dt2 * Kz[g];
    if (gv0) gv0[g] = -dt * gm1;
  }
}


// y = m x entry-wise (a lumped mass applied; no Dirichlet treatment).
static __global__ void __launch_bounds__(kVecThreads) k_diag_mul(int64_t n, const double* __restrict__ m,
                                                                 const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    y[g] = m[g] * x[g];
}

// x = b / m on free DOFs, 0 on constrained ones (a lumped mass solved).
static __global__ void __launch_bounds__(kVecThreads) k_lumped_solve(MeshInfo mi, const double* __restrict__ m,
                                                                     const double* __restrict__ b,
                                                                     double* __restrict__ x) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x)
    x[g] = dof_constrained(mi, g) ? 0.0 : b[g] / m[g];
}

// One central-difference step with a lumped mass (Sec. 4.1, eq. Motion_explicit2):
// a = (P - R) / m and u_prev <- 2 u - u_prev + dt^2 a on free DOFs; a = 0 and
// u_prev <- u on constrained ones.
static __global__ void __launch_bounds__(kVecThreads) k_cd_lumped(MeshInfo mi, const double* __restrict__ u,
                                                                  const double* __restrict__ Pl,
                                                                  const double* __restrict__ R,
                                                                  const double* __restrict__ m, double dt2,
                                                                  double* __restrict__ a,
                                                                  double* __restrict__ u_prev) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x) {
    const double un = u[g];
    if (dof_constrained(mi, g)) {
      a[g] = 0.0;
      u_prev[g] = un;
    } else {
      const double ag = (Pl[g] - R[g]) / m[g];
      a[g] = ag;
      u_prev[g] = 2.0 * un - u_prev[g] + dt2 * ag;
    }
  }
}

}  // namespace sdme
