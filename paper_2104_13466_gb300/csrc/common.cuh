// Device helpers shared by the element and vector kernels: reductions,
// the last-CTA-done pattern and the PCG scalar block.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sdme {

// Linearisation state layout per element: [10][Q^3]: H = F^{-T} (9, row
// major iJ) then c = mu - lambda ln J.  The float32 copy holds
// Ht_cd = sqrt(w_q detJ) s_d H_cd in place of H (w_q the product of the
// Gauss weights, s_d = 2 / h_d), so that the quadrature weight and the
// reference-to-physical derivative scales fold into the tangent action.
constexpr int kStateFields = 10;

// PCG status values held in PcgScalars::status
constexpr int kPcgRunning = 0;
constexpr int kPcgConverged = 1;
constexpr int kPcgMaxit = 2;
constexpr int kPcgBreakdown = 3;   // non-positive or non-finite curvature / residual

// Scalars of one Jacobi-PCG solve, resident in device memory so that an
// iteration needs no host round trip.  All float64.
struct PcgScalars {
  double rz;       // r . z of the current iterate
  double pq;       // p . (A p)
  double rr;       // r . r
  double bb;       // b . b (of the scaled right-hand side)
  double alpha, beta;
  double tol2;     // rtol^2 * bb
  int iter, maxit;
  int status;
  unsigned int counter;   // last-CTA counters (reset by the finishing CTA)
  unsigned int counter2;
  int pad;
};

// Lattice description used by per-DOF kernels.
struct MeshInfo {
  int N[3];
  int64_t Nn;
  int64_t ndof;
  unsigned clamp[6];
};

__device__ __forceinline__ bool dof_constrained(const MeshInfo& m, int64_t g) {
  const int c = (int)(g / m.Nn);
  const int64_t r = g - (int64_t)c * m.Nn;
  const int ix = (int)(r % m.N[0]);
  const int64_t t = r / m.N[0];
  const int iy = (int)(t % m.N[1]);
  const int iz = (int)(t / m.N[1]);
  const unsigned bit = 1u << c;
  return ((ix == 0) && (m.clamp[0] & bit)) || ((ix == m.N[0] - 1) && (m.clamp[1] & bit)) ||
         ((iy == 0) && (m.clamp[2] & bit)) || ((iy == m.N[1] - 1) && (m.clamp[3] & bit)) ||
         ((iz == 0) && (m.clamp[4] & bit)) || ((iz == m.N[2] - 1) && (m.clamp[5] & bit));
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// the programmatic-serialization attribute may start while its predecessor
// in the stream still runs: pdl_wait() returns once the predecessor grid has
// completed and its memory operations are visible (at once for a normal
// launch), and pdl_trigger() lets the successor start launching once every
// CTA has issued it or exited.  A kernel reads nothing its predecessor writes
// before pdl_wait().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Per-thread partial sums of float32 terms.  A compensated (float-float)
// accumulator: s + c carries the running sum to about 48 bits with float32
// adds only (Knuth's TwoSum gives each addition's rounding error exactly,
// collected in c), as accurate as a float64 accumulator of the same float32
// terms; on GB300 the float64 pipe runs a small fraction of the float32 rate
// and a float64 add per term kept the PCG update kernel float64-bound.
struct FFSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    c = __fadd_rn(c, err);
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// s + c += s2 + c2 (TwoSum of the leading words, the low words added):
// commutative, so a butterfly reduction leaves the same pair in every lane.
__device__ __forceinline__ void ff_merge(float& s, float& c, float s2, float c2) {
  const float t = __fadd_rn(s, s2);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
  s = t;
  c = __fadd_rn(__fadd_rn(c, c2), err);
}

// Accumulator of TV terms: FFSum for float32, plain float64 for float64.
template <typename TV>
struct AccOf {
  struct type {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ double value() const { return v; }
  };
};
template <>
struct AccOf<float> {
  using type = FFSum;
};

// Sum over the CTA (float64); result valid in every thread.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red_[32];
  __shared__ double out_;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red_[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = (threadIdx.x < ((blockDim.x + 31) >> 5)) ? red_[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) out_ = w;
  }
  __syncthreads();
  return out_;
}

// Sum over the CTA in the given type; result valid in every thread.
template <typename T>
__device__ __forceinline__ T block_sum_t(T v) {
  __shared__ T red_t_[32];
  __shared__ T out_t_;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red_t_[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    T w = (threadIdx.x < ((blockDim.x + 31) >> 5)) ? red_t_[threadIdx.x] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) out_t_ = w;
  }
  __syncthreads();
  return out_t_;
}

// Two CTA sums of compensated float32 partials, in float64 in every thread:
// the warps reduce their pairs with float32 adds (ff_merge), and only the
// per-warp totals go through the float64 pipe.
__device__ __forceinline__ void block_sum2_ff(const FFSum& a, const FFSum& b, double& oa, double& ob) {
  __shared__ double fa_[32], fb_[32];
  __shared__ double foa_, fob_;
  float as = a.s, ac = a.c, bs = b.s, bc = b.c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float as2 = __shfl_xor_sync(0xffffffffu, as, o), ac2 = __shfl_xor_sync(0xffffffffu, ac, o);
    const float bs2 = __shfl_xor_sync(0xffffffffu, bs, o), bc2 = __shfl_xor_sync(0xffffffffu, bc, o);
    ff_merge(as, ac, as2, ac2);
    ff_merge(bs, bc, bs2, bc2);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    fa_[threadIdx.x >> 5] = (double)as + (double)ac;
    fb_[threadIdx.x >> 5] = (double)bs + (double)bc;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool ok = threadIdx.x < ((blockDim.x + 31) >> 5);
    double x = ok ? fa_[threadIdx.x] : 0.0, y = ok ? fb_[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (threadIdx.x == 0) {
      foa_ = x;
      fob_ = y;
    }
  }
  __syncthreads();
  oa = foa_;
  ob = fob_;
}

// CTA sum of compensated float32 partials in float64, valid in every thread
// (as block_sum2_ff, one value).
__device__ __forceinline__ double block_sum_ff(const FFSum& a) {
  __shared__ double fr_[32];
  __shared__ double fo_;
  float as = a.s, ac = a.c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float as2 = __shfl_xor_sync(0xffffffffu, as, o), ac2 = __shfl_xor_sync(0xffffffffu, ac, o);
    ff_merge(as, ac, as2, ac2);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) fr_[threadIdx.x >> 5] = (double)as + (double)ac;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = (threadIdx.x < ((blockDim.x + 31) >> 5)) ? fr_[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (threadIdx.x == 0) fo_ = x;
  }
  __syncthreads();
  return fo_;
}

// Two sums at once.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double ra_[32], rb_[32];
  __shared__ double oa_, ob_;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    ra_[threadIdx.x >> 5] = a;
    rb_[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool ok = threadIdx.x < ((blockDim.x + 31) >> 5);
    double x = ok ? ra_[threadIdx.x] : 0.0, y = ok ? rb_[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (threadIdx.x == 0) {
      oa_ = x;
      ob_ = y;
    }
  }
  __syncthreads();
  a = oa_;
  b = ob_;
}

// Call after thread 0 of every CTA has written its partial(s).  Returns
// true in every thread of the last CTA to arrive; that CTA must reset the
// counter.  Nothing waits: CTAs that are not last simply return false.
__device__ __forceinline__ bool last_block_done(unsigned int* counter) {
  __shared__ bool last_;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    last_ = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last_) __threadfence();
  return last_;
}

// As last_block_done, for `total` arrivals that need not equal the grid
// size (several problems per launch, or CTAs looping over elements).
__device__ __forceinline__ bool last_arrival(unsigned int* counter, unsigned int total) {
  __shared__ bool last_a_;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    last_a_ = (t == total - 1);
  }
  __syncthreads();
  if (last_a_) __threadfence();
  return last_a_;
}

// Deterministic sum of m partials (fixed strided order + fixed tree).
__device__ __forceinline__ double ordered_sum(const double* part, int m) {
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += ((const volatile double*)part)[i];
  return block_sum(s);
}

// Deterministic sum of m partials written by an earlier kernel, with eight
// loads in flight per thread (fixed order for a given m and block size).
__device__ __forceinline__ double ordered_sum_prev(const double* __restrict__ part, int m) {
  const int bd = blockDim.x;
  double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int i = threadIdx.x;
  for (; i + 7 * bd < m; i += 8 * bd) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] += __ldcg(part + i + k * bd);
  }
  for (; i < m; i += bd) a[0] += __ldcg(part + i);
  return block_sum(((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7])));
}

}  // namespace sdme
