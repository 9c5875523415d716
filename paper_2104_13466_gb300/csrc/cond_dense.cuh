// Static condensation of the element-interior modes (float64): per-element
// dense factorisation of the interior block and the element Schur
// complements, and the operators of the condensed Jacobi-PCG.
//
// Per element e (local DOF sets: interior I, |I| = Ni; skeleton B, |B| = Nb;
// the masked element matrix A = Ke[e] from cond_columns_kernel):
//   L L^T = A_II (Cholesky),   W = L^{-1} A_IB,   S_e = A_BB - W^T W,
//   condensed right-hand side  g_B = f_B - W^T (L^{-1} f_I),
//   interior recovery          x_I = L^{-T} (L^{-1} f_I - W x_B).
// Layouts: Ke[e] column-major N x N (N = Ni + Nb); L[e] row-major Ni x Ni;
// W[e] row-major Ni x Nb; S[e] row-major Nb x Nb; Y[e] = L^{-1} f_I.
// gI[e][i], gB[e][b]: global DOF of the element's interior / skeleton entry
// (gB = -1 for a constrained DOF: its row and column of S_e are zero).
#pragma once

#include "common.cuh"

namespace sdme {

constexpr int kCondThreads = 512;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// L = chol(A_II); err[e] = 1 if A_II is not positive definite.
static __global__ void __launch_bounds__(kCondThreads) cond_factor_kernel(int N, int Ni, const int* __restrict__ Il,
                                                                        const double* __restrict__ Ke,
                                                                        double* __restrict__ L, int* err) {
  const int e = blockIdx.x;
  const double* A = Ke + (int64_t)e * N * N;
  double* Le = L + (int64_t)e * Ni * Ni;
  for (int t = threadIdx.x; t < Ni * Ni; t += blockDim.x) {
    const int i = t / Ni, k = t - i * Ni;
    Le[t] = A[(int64_t)Il[k] * N + Il[i]];
  }
  __syncthreads();
  __shared__ double dk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < Ni; ++k) {
    double s = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) s += Le[k * Ni + j] * Le[k * Ni + j];
    s = block_sum(s);
    if (threadIdx.x == 0) {
      double a = Le[k * Ni + k] - s;
      if (!(a > 0.0)) {
        err[e] = 1;
        a = 1.0;
      }
      dk = sqrt(a);
      Le[k * Ni + k] = dk;
    }
    __syncthreads();
    const double inv = 1.0 / dk;
    for (int i = k + 1 + warp; i < Ni; i += nw) {
      double dot = 0.0;
      for (int j = lane; j < k; j += 32) dot += Le[i * Ni + j] * Le[k * Ni + j];
      dot = warp_sum(dot);
      if (lane == 0) Le[i * Ni + k] = (Le[i * Ni + k] - dot) * inv;
    }
    __syncthreads();
  }
}

// W = L^{-1} A_IB (forward substitution, one thread per skeleton column).
static __global__ void __launch_bounds__(kCondThreads) cond_trsm_kernel(int N, int Ni, int Nb,
                                                                      const int* __restrict__ Il,
                                                                      const int* __restrict__ Bl,
                                                                      const double* __restrict__ Ke,
                                                                      const double* __restrict__ L,
                                                                      double* __restrict__ W) {
  const int e = blockIdx.x;
  const double* A = Ke + (int64_t)e * N * N;
  const double* Le = L + (int64_t)e * Ni * Ni;
  double* We = W + (int64_t)e * Ni * Nb;
  for (int b = threadIdx.x; b < Nb; b += blockDim.x) {
    const double* col = A + (int64_t)Bl[b] * N;
    for (int i = 0; i < Ni; ++i) {
      double v = col[Il[i]];
      for (int k = 0; k < i; ++k) v -= Le[i * Ni + k] * We[(int64_t)k * Nb + b];
      We[(int64_t)i * Nb + b] = v / Le[i * Ni + i];
    }
  }
}

// S_e = A_BB - W^T W (32 x 32 output tiles; grid (tiles, tiles, elements)).
static __global__ void __launch_bounds__(1024) cond_syrk_kernel(int N, int Ni, int Nb, const int* __restrict__ Bl,
                                                              const double* __restrict__ Ke,
                                                              const double* __restrict__ W,
                                                              double* __restrict__ S) {
  const int e = blockIdx.z;
  const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
  const int ty = threadIdx.y, tx = threadIdx.x;
  const double* We = W + (int64_t)e * Ni * Nb;
  __shared__ double Ta[32][33], Tb[32][33];
  double acc = 0.0;
  for (int i0 = 0; i0 < Ni; i0 += 32) {
    const int i = i0 + ty;
    Ta[ty][tx] = (i < Ni && a0 + tx < Nb) ? We[(int64_t)i * Nb + a0 + tx] : 0.0;
    Tb[ty][tx] = (i < Ni && b0 + tx < Nb) ? We[(int64_t)i * Nb + b0 + tx] : 0.0;
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) acc += Ta[k][ty] * Tb[k][tx];
    __syncthreads();
  }
  const int a = a0 + ty, b = b0 + tx;
  if (a < Nb && b < Nb) {
    const double abb = Ke[(int64_t)e * N * N + (int64_t)Bl[b] * N + Bl[a]];
    S[(int64_t)e * Nb * Nb + (int64_t)a * Nb + b] = abb - acc;
  }
}

// y += sum_e S_e x_B (skeleton DOFs); with partial/scal, the PCG step length
// from p.q = sum_e x_B . S_e x_B, finished by the last element CTA.
static __global__ void __launch_bounds__(256) cond_apply_kernel(int Nb, const int64_t* __restrict__ gB,
                                                              const double* __restrict__ S,
                                                              const double* __restrict__ x, double* __restrict__ y,
                                                              double* __restrict__ partial, PcgScalars* scal) {
  if (scal && scal->status != kPcgRunning) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* xb = reinterpret_cast<double*>(smem_raw);
  const int e = blockIdx.x;
  const int64_t* g = gB + (int64_t)e * Nb;
  for (int b = threadIdx.x; b < Nb; b += blockDim.x) xb[b] = g[b] >= 0 ? x[g[b]] : 0.0;
  __syncthreads();
  const double* Se = S + (int64_t)e * Nb * Nb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double dot = 0.0;
  for (int a = warp; a < Nb; a += nw) {
    double v = 0.0;
    for (int b = lane; b < Nb; b += 32) v += Se[(int64_t)a * Nb + b] * xb[b];
    v = warp_sum(v);
    if (lane == 0 && g[a] >= 0) {
      atomicAdd(&y[g[a]], v);
      dot += xb[a] * v;
    }
  }
  if (partial) {
    const double tot = block_sum(dot);
    if (threadIdx.x == 0) partial[e] = tot;
    if (scal && last_arrival(&scal->counter, gridDim.x)) {
      const double pq = ordered_sum(partial, gridDim.x);
      if (threadIdx.x == 0) {
        scal->pq = pq;
        scal->alpha = scal->rz / pq;
        if (!(pq > 0.0) || !isfinite(scal->alpha)) scal->status = kPcgBreakdown;
        scal->counter = 0;
      }
    }
  }
}

// d += diag(S_e) on the skeleton DOFs.
static __global__ void __launch_bounds__(256) cond_diag_kernel(int Nb, const int64_t* __restrict__ gB,
                                                             const double* __restrict__ S, double* __restrict__ d) {
  const int e = blockIdx.x;
  for (int b = threadIdx.x; b < Nb; b += blockDim.x) {
    const int64_t gg = gB[(int64_t)e * Nb + b];
    if (gg >= 0) atomicAdd(&d[gg], S[(int64_t)e * Nb * Nb + (int64_t)b * Nb + b]);
  }
}

// g = f on free skeleton DOFs, 0 on interior and constrained ones; interior
// entries of d set to 1 (they never enter the condensed iteration).
static __global__ void __launch_bounds__(256) cond_rhs_init(MeshInfo mi, int P, const double* __restrict__ f,
                                                                      double* __restrict__ g, double* __restrict__ d) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < mi.ndof; k += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(k / mi.Nn);
    const int64_t r = k - (int64_t)c * mi.Nn;
    const int ix = (int)(r % mi.N[0]);
    const int64_t t = r / mi.N[0];
    const int iy = (int)(t % mi.N[1]), iz = (int)(t / mi.N[1]);
    const bool inner = (ix % P != 0) && (iy % P != 0) && (iz % P != 0);
    g[k] = (inner || dof_constrained(mi, k)) ? 0.0 : f[k];
    if (d && inner) d[k] = 1.0;
  }
}

// Y_e = L^{-1} f_I (one warp, forward substitution), then g_B -= W^T Y_e.
static __global__ void __launch_bounds__(256) cond_rhs_kernel(int Ni, int Nb, const int64_t* __restrict__ gI,
                                                            const int64_t* __restrict__ gB,
                                                            const double* __restrict__ L,
                                                            const double* __restrict__ W,
                                                            const double* __restrict__ f, double* __restrict__ g,
                                                            double* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* ys = reinterpret_cast<double*>(smem_raw);
  const int e = blockIdx.x;
  const double* Le = L + (int64_t)e * Ni * Ni;
  const double* We = W + (int64_t)e * Ni * Nb;
  for (int i = threadIdx.x; i < Ni; i += blockDim.x) ys[i] = f[gI[(int64_t)e * Ni + i]];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = 0; i < Ni; ++i) {
      double dot = 0.0;
      for (int k = lane; k < i; k += 32) dot += Le[i * Ni + k] * ys[k];
      dot = warp_sum(dot);
      if (lane == 0) ys[i] = (ys[i] - dot) / Le[i * Ni + i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < Ni; i += blockDim.x) Y[(int64_t)e * Ni + i] = ys[i];
  for (int b = threadIdx.x; b < Nb; b += blockDim.x) {
    const int64_t gg = gB[(int64_t)e * Nb + b];
    if (gg < 0) continue;
    double v = 0.0;
    for (int i = 0; i < Ni; ++i) v += We[(int64_t)i * Nb + b] * ys[i];
    atomicAdd(&g[gg], -v);
  }
}

// x_I = L^{-T} (Y_e - W x_B) (rows of W by warps, one warp for the
// backward substitution); interior DOFs belong to one element only.
static __global__ void __launch_bounds__(256) cond_recover_kernel(int Ni, int Nb, const int64_t* __restrict__ gI,
                                                                const int64_t* __restrict__ gB,
                                                                const double* __restrict__ L,
                                                                const double* __restrict__ W,
                                                                const double* __restrict__ Y, double* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* xb = reinterpret_cast<double*>(smem_raw);
  double* t = xb + Nb;
  const int e = blockIdx.x;
  const double* Le = L + (int64_t)e * Ni * Ni;
  const double* We = W + (int64_t)e * Ni * Nb;
  const int64_t* gb = gB + (int64_t)e * Nb;
  for (int b = threadIdx.x; b < Nb; b += blockDim.x) xb[b] = gb[b] >= 0 ? x[gb[b]] : 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < Ni; i += nw) {
    double v = 0.0;
    for (int b = lane; b < Nb; b += 32) v += We[(int64_t)i * Nb + b] * xb[b];
    v = warp_sum(v);
    if (lane == 0) t[i] = Y[(int64_t)e * Ni + i] - v;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int i = Ni - 1; i >= 0; --i) {
      double dot = 0.0;
      for (int k = i + 1 + lane; k < Ni; k += 32) dot += Le[k * Ni + i] * t[k];
      dot = warp_sum(dot);
      if (lane == 0) t[i] = (t[i] - dot) / Le[i * Ni + i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < Ni; i += blockDim.x) x[gI[(int64_t)e * Ni + i]] = t[i];
}

}  // namespace sdme
