// Sum-factorised, matrix-free element kernels for tensor-product hexahedra.
//
// One CTA per element.  The element's (P+1)^3 x 3 coefficients are gathered
// from the global lattice, taken to the Q^3 Gauss points (Q = P + 2) by three
// 1D contractions with B[q][p] = phi_p(xi_q) (eq. ProdTensorialHexaedro
// applied one direction at a time), differentiated along each direction
// with the collocation-derivative matrix DQ on the Gauss points (exact for
// the degree-P restriction of u to each line), combined pointwise in
// registers, and taken back by the transposed stages before an atomic
// scatter-add to the global vector.
//
// Shared memory (T words): U[3][Q^3] (values / value fluxes) and
// G[9][Q^3] (gradients / stress fluxes).  Gather and the intermediate
// interpolation buffers alias the G region while G is not live.
//
// The 1D tables travel in the kernel parameter block (__grid_constant__),
// so the fully unrolled contractions read them as constant-bank operands.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace sdme {

template <typename T, int P>
struct ElemTables {
  static constexpr int n = P + 1;
  static constexpr int Q = P + 2;
  T B[Q * n];   // B[q*n + p] = phi_p(xi_q), lattice order
  T D[Q * n];   // D[q*n + p] = phi_p'(xi_q)
  T DQ[Q * Q];  // DQ[q*Q + m] = l_m'(xi_q), Lagrange through the Gauss points
  T W[Q];       // Gauss weights
};

template <typename T, int P>
struct ElemParams {
  ElemTables<T, P> tab;
  T s[3];        // 2 / h_d: reference-to-physical derivative scale
  T detJ;        // h_x h_y h_z / 8
  T mu, lam, rho;
  T b1;          // coefficient of the mass term fused into the operator
  int ne[3];     // elements per direction
  int N[3];      // lattice points per direction
  int64_t Nn;    // lattice points (per component)
  unsigned clamp[6];
};

// Lattice point on a clamped face for component c?
template <typename Prm>
__device__ __forceinline__ bool is_constrained(const Prm& p, int c, int ix, int iy, int iz) {
  const unsigned bit = 1u << c;
  return ((ix == 0) && (p.clamp[0] & bit)) || ((ix == p.N[0] - 1) && (p.clamp[1] & bit)) ||
         ((iy == 0) && (p.clamp[2] & bit)) || ((iy == p.N[1] - 1) && (p.clamp[3] & bit)) ||
         ((iz == 0) && (p.clamp[4] & bit)) || ((iz == p.N[2] - 1) && (p.clamp[5] & bit));
}

// Contract a set of 3D arrays along one axis, one thread per line.
// Arrays are [d2][d1][d0] (d0 fastest); a line runs along the contracted
// axis, whose extent goes NI -> NO.  `outer` = product of the extents before
// the axis, `inner` = product after it (stride of the axis).  Fields are
// `sfs` / `dfs` words apart.  Matrix: !TR: out[o] = sum_i M[o*NI + i] in[i];
// TR: out[o] = sum_i M[i*NO + o] in[i].  ACC adds into dst.
template <int NI, int NO, bool TR, bool ACC, typename T>
__device__ __forceinline__ void contract(const T* __restrict__ src, T* __restrict__ dst,
                                         const T* __restrict__ M, int nfields, int outer, int inner,
                                         int sfs, int dfs) {
  const int per_field = outer * inner;
  const int total = nfields * per_field;
  for (int l = threadIdx.x; l < total; l += blockDim.x) {
    const int f = l / per_field;
    const int rem = l - f * per_field;
    const int o = rem / inner;
    const int i = rem - o * inner;
    const T* s = src + f * sfs + o * NI * inner + i;
    T* d = dst + f * dfs + o * NO * inner + i;
    T in[NI];
#pragma unroll
    for (int a = 0; a < NI; ++a) in[a] = s[a * inner];
#pragma unroll
    for (int b = 0; b < NO; ++b) {
      T acc = ACC ? d[b * inner] : T(0);
#pragma unroll
      for (int a = 0; a < NI; ++a) acc += (TR ? M[a * NO + b] : M[b * NI + a]) * in[a];
      d[b * inner] = acc;
    }
  }
}

// Forward: X[3][n^3] (in Gb region) -> U[3][Q^3] values.  Buffers:
// S1 = [3][n][n][Q], S2 = [3][n][Q][Q], placed after X inside Gb.
template <typename T, int P>
__device__ __forceinline__ void interp_forward(const ElemTables<T, P>& tb, T* X, T* U, T* Gb) {
  constexpr int n = P + 1, Q = P + 2;
  T* S1 = Gb + 3 * n * n * n;
  T* S2 = S1 + 3 * n * n * Q;
  contract<n, Q, false, false>(X, S1, tb.B, 3, n * n, 1, n * n * n, n * n * Q);
  __syncthreads();
  contract<n, Q, false, false>(S1, S2, tb.B, 3, n, Q, n * n * Q, n * Q * Q);
  __syncthreads();
  contract<n, Q, false, false>(S2, U, tb.B, 3, 1, Q * Q, n * Q * Q, Q * Q * Q);
  __syncthreads();
}

// Collocated reference derivatives: G[(c*3+d)][Q^3] = d/dxi_d U_c.
template <typename T, int P>
__device__ __forceinline__ void derivs_forward(const ElemTables<T, P>& tb, const T* U, T* G) {
  constexpr int Q = P + 2, Q3 = Q * Q * Q;
  contract<Q, Q, false, false>(U, G + 0 * Q3, tb.DQ, 3, Q * Q, 1, Q3, 3 * Q3);
  contract<Q, Q, false, false>(U, G + 1 * Q3, tb.DQ, 3, Q, Q, Q3, 3 * Q3);
  contract<Q, Q, false, false>(U, G + 2 * Q3, tb.DQ, 3, 1, Q * Q, Q3, 3 * Q3);
  __syncthreads();
}

// Transposed derivatives accumulated into the value fluxes:
// U_c += sum_d DQ_d^T G_cd.
template <typename T, int P>
__device__ __forceinline__ void derivs_transpose(const ElemTables<T, P>& tb, const T* G, T* U) {
  constexpr int Q = P + 2, Q3 = Q * Q * Q;
  contract<Q, Q, true, true>(G + 0 * Q3, U, tb.DQ, 3, Q * Q, 1, 3 * Q3, Q3);
  __syncthreads();
  contract<Q, Q, true, true>(G + 1 * Q3, U, tb.DQ, 3, Q, Q, 3 * Q3, Q3);
  __syncthreads();
  contract<Q, Q, true, true>(G + 2 * Q3, U, tb.DQ, 3, 1, Q * Q, 3 * Q3, Q3);
  __syncthreads();
}

// Transposed interpolation U[3][Q^3] -> Y[3][n^3] (Y at the start of Gb).
template <typename T, int P>
__device__ __forceinline__ void interp_transpose(const ElemTables<T, P>& tb, const T* U, T* Gb) {
  constexpr int n = P + 1, Q = P + 2;
  T* Y = Gb;
  T* S1 = Gb + 3 * n * n * n;
  T* S2 = S1 + 3 * n * n * Q;
  contract<Q, n, true, false>(U, S2, tb.B, 3, 1, Q * Q, Q * Q * Q, n * Q * Q);
  __syncthreads();
  contract<Q, n, true, false>(S2, S1, tb.B, 3, n, Q, n * Q * Q, n * n * Q);
  __syncthreads();
  contract<Q, n, true, false>(S1, Y, tb.B, 3, n * n, 1, n * n * Q, n * n * n);
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ double to_double(T v) { return static_cast<double>(v); }

// element index -> (ex, ey, ez); local (c, m) -> global DOF; constrained?
template <typename Prm>
__device__ __forceinline__ int64_t dof_index(const Prm& p, int P, int ex, int ey, int ez, int idx,
                                             bool* cons) {
  const int n = P + 1, n3 = n * n * n;
  const int c = idx / n3;
  const int m = idx - c * n3;
  const int r = m / (n * n);
  const int q = (m / n) % n;
  const int pp = m % n;
  const int ix = ex * P + pp, iy = ey * P + q, iz = ez * P + r;
  *cons = is_constrained(p, c, ix, iy, iz);
  return c * p.Nn + ((int64_t)iz * p.N[1] + iy) * (int64_t)p.N[0] + ix;
}

template <typename T>
__device__ __forceinline__ T wprod(const T* W, int q, int Q) {
  const int k1 = q % Q, k2 = (q / Q) % Q, k3 = q / (Q * Q);
  return W[k1] * W[k2] * W[k3];
}

// Number of threads per CTA for order P.
__host__ __device__ constexpr int elem_threads(int P) {
  return ((P + 2) * (P + 2) * (P + 2) + 31) / 32 * 32 > 512 ? 512
                                                            : ((P + 2) * (P + 2) * (P + 2) + 31) / 32 * 32;
}

template <int P>
constexpr int elem_smem_words() {
  return 12 * (P + 2) * (P + 2) * (P + 2);
}


//-----------------------------------------------------------------------------
// Residual: y += R(u) + b1 M u, and the linearisation state at u.
// Internal force = int P(F) : grad N dV, P = mu (F - F^{-T}) + lambda ln J F^{-T}
// (first Piola form of eq. second Piolla_Kirchhoff relation).
//-----------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(elem_threads(P))
residual_kernel(const __grid_constant__ ElemParams<double, P> prm, const double* __restrict__ u,
                double* __restrict__ y, double* __restrict__ st64, float* __restrict__ st32,
                int* __restrict__ err) {
  using T = double;
  constexpr int n = P + 1, Q = P + 2, n3 = n * n * n, Q3 = Q * Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* U = reinterpret_cast<T*>(smem_raw);
  T* G = U + 3 * Q3;
  const int e = blockIdx.x;
  const int ex = e % prm.ne[0], ey = (e / prm.ne[0]) % prm.ne[1], ez = e / (prm.ne[0] * prm.ne[1]);
  for (int idx = threadIdx.x; idx < 3 * n3; idx += blockDim.x) {
    bool cons;
    int64_t g = dof_index(prm, P, ex, ey, ez, idx, &cons);
    G[idx] = u[g];
  }
  __syncthreads();
  interp_forward<T, P>(prm.tab, G, U, G);
  derivs_forward<T, P>(prm.tab, U, G);
  const T s0 = prm.s[0], s1 = prm.s[1], s2 = prm.s[2];
  const T sc[3] = {s0, s1, s2};
  for (int q = threadIdx.x; q < Q3; q += blockDim.x) {
    T F[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) F[c][d] = (c == d ? T(1) : T(0)) + G[(c * 3 + d) * Q3 + q] * sc[d];
    T cof[3][3];
    cof[0][0] = F[1][1] * F[2][2] - F[1][2] * F[2][1];
    cof[0][1] = F[1][2] * F[2][0] - F[1][0] * F[2][2];
    cof[0][2] = F[1][0] * F[2][1] - F[1][1] * F[2][0];
    cof[1][0] = F[0][2] * F[2][1] - F[0][1] * F[2][2];
    cof[1][1] = F[0][0] * F[2][2] - F[0][2] * F[2][0];
    cof[1][2] = F[0][1] * F[2][0] - F[0][0] * F[2][1];
    cof[2][0] = F[0][1] * F[1][2] - F[0][2] * F[1][1];
    cof[2][1] = F[0][2] * F[1][0] - F[0][0] * F[1][2];
    cof[2][2] = F[0][0] * F[1][1] - F[0][1] * F[1][0];
    const T J = F[0][0] * cof[0][0] + F[0][1] * cof[0][1] + F[0][2] * cof[0][2];
    if (!(J > T(0))) atomicOr(err, 1);
    const T iJ = T(1) / J;
    const T lnJ = log(J);
    const T wdet = wprod(prm.tab.W, q, Q) * prm.detJ;
    const T a = prm.lam * lnJ;
    const T cst = prm.mu - a;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T H = cof[c][d] * iJ;  // (F^{-T})_cd
        const T Pcd = prm.mu * (F[c][d] - H) + a * H;
        G[(c * 3 + d) * Q3 + q] = wdet * Pcd * sc[d];
        const int64_t so = ((int64_t)e * kStateFields + (c * 3 + d)) * Q3 + q;
        if (st64) st64[so] = H;
        if (st32) st32[so] = (float)H;
      }
    const int64_t so = ((int64_t)e * kStateFields + 9) * Q3 + q;
    if (st64) st64[so] = cst;
    if (st32) st32[so] = (float)cst;
    const T mfac = prm.b1 * prm.rho * wdet;
#pragma unroll
    for (int c = 0; c < 3; ++c) U[c * Q3 + q] *= mfac;
  }
  __syncthreads();
  derivs_transpose<T, P>(prm.tab, G, U);
  interp_transpose<T, P>(prm.tab, U, G);
  for (int idx = threadIdx.x; idx < 3 * n3; idx += blockDim.x) {
    bool cons;
    int64_t g = dof_index(prm, P, ex, ey, ez, idx, &cons);
    atomicAdd(&y[g], G[idx]);
  }
}

//-----------------------------------------------------------------------------
// Tangent: y += (b1 M + K_T(u)) x on free DOFs (x taken as 0 on constrained
// DOFs), and dot_out[e] = x_e . (K_e x_e) for the PCG step length.
// dP = mu dF + c F^{-T} dF^T F^{-T} + lambda (F^{-T} : dF) F^{-T}, c = mu - lambda ln J
// (consistent linearisation of the first Piola stress, Sec. 3).
// T: arithmetic type; TV: global vector type; TS: stored-state type.
//-----------------------------------------------------------------------------
template <int P, typename T, typename TV>
__global__ void __launch_bounds__(elem_threads(P))
tangent_kernel(const __grid_constant__ ElemParams<T, P> prm, const TV* __restrict__ x,
               TV* __restrict__ y, const T* __restrict__ st, double* __restrict__ dot_partial,
               PcgScalars* __restrict__ scal) {
  constexpr int n = P + 1, Q = P + 2, n3 = n * n * n, Q3 = Q * Q * Q;
  if (scal && scal->status != 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* U = reinterpret_cast<T*>(smem_raw);
  T* G = U + 3 * Q3;
  const int e = blockIdx.x;
  const int ex = e % prm.ne[0], ey = (e / prm.ne[0]) % prm.ne[1], ez = e / (prm.ne[0] * prm.ne[1]);
  for (int idx = threadIdx.x; idx < 3 * n3; idx += blockDim.x) {
    bool cons;
    int64_t g = dof_index(prm, P, ex, ey, ez, idx, &cons);
    G[idx] = cons ? T(0) : (T)x[g];
  }
  __syncthreads();
  interp_forward<T, P>(prm.tab, G, U, G);
  derivs_forward<T, P>(prm.tab, U, G);
  const T sc[3] = {prm.s[0], prm.s[1], prm.s[2]};
  const T* ste = st + (int64_t)e * kStateFields * Q3;
  for (int q = threadIdx.x; q < Q3; q += blockDim.x) {
    T H[3][3], dF[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        H[c][d] = ste[(c * 3 + d) * Q3 + q];
        dF[c][d] = G[(c * 3 + d) * Q3 + q] * sc[d];
      }
    const T cst = ste[9 * Q3 + q];
    T tr = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) tr += H[c][d] * dF[c][d];
    // W = dF^T H ; V = H W
    T W[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < 3; ++j) W[a][j] = dF[0][a] * H[0][j] + dF[1][a] * H[1][j] + dF[2][a] * H[2][j];
    const T wdet = wprod(prm.tab.W, q, Q) * prm.detJ;
    const T ltr = prm.lam * tr;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const T V = H[i][0] * W[0][j] + H[i][1] * W[1][j] + H[i][2] * W[2][j];
        const T dP = prm.mu * dF[i][j] + cst * V + ltr * H[i][j];
        G[(i * 3 + j) * Q3 + q] = wdet * dP * sc[j];
      }
    const T mfac = prm.b1 * prm.rho * wdet;
#pragma unroll
    for (int c = 0; c < 3; ++c) U[c * Q3 + q] *= mfac;
  }
  __syncthreads();
  derivs_transpose<T, P>(prm.tab, G, U);
  interp_transpose<T, P>(prm.tab, U, G);
  T dotT = T(0);
  for (int idx = threadIdx.x; idx < 3 * n3; idx += blockDim.x) {
    bool cons;
    int64_t g = dof_index(prm, P, ex, ey, ez, idx, &cons);
    if (!cons) {
      const T v = G[idx];
      atomicAdd(&y[g], (TV)v);
      if (dot_partial) dotT += v * (T)x[g];
    }
  }
  if (dot_partial) {
    // x_e . (K_e x_e) summed over elements gives x . (K x) for the PCG step
    // length; float64 across threads, fixed-order (deterministic) finalize
    // by the last CTA to finish.
    const double tot = block_sum(static_cast<double>(dotT));
    if (threadIdx.x == 0) dot_partial[e] = tot;
    if (scal && last_block_done(&scal->counter)) {
      const double pq = ordered_sum(dot_partial, gridDim.x);
      if (threadIdx.x == 0) {
        scal->pq = pq;
        scal->alpha = scal->rz / pq;
        if (!(pq > 0.0) || !isfinite(scal->alpha)) scal->status = kPcgBreakdown;
        scal->counter = 0;
      }
    }
  }
}

//-----------------------------------------------------------------------------
// Mass: y += M x (no Dirichlet treatment).
//-----------------------------------------------------------------------------
template <int P, typename T>
__global__ void __launch_bounds__(elem_threads(P))
mass_kernel(const __grid_constant__ ElemParams<T, P> prm, const double* __restrict__ x,
            double* __restrict__ y) {
  constexpr int n = P + 1, Q = P + 2, n3 = n * n * n, Q3 = Q * Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* U = reinterpret_cast<T*>(smem_raw);
  T* G = U + 3 * Q3;
  const int e = blockIdx.x;
  const int ex = e % prm.ne[0], ey = (e / prm.ne[0]) % prm.ne[1], ez = e / (prm.ne[0] * prm.ne[1]);
  for (int idx = threadIdx.x; idx < 3 * n3; idx += blockDim.x) {
    bool cons;
    int64_t g = dof_index(prm, P, ex, ey, ez, idx, &cons);
    G[idx] = (T)x[g];
  }
  __syncthreads();
  interp_forward<T, P>(prm.tab, G, U, G);
  for (int q = threadIdx.x; q < Q3; q += blockDim.x) {
    const T f = prm.rho * wprod(prm.tab.W, q, Q) * prm.detJ;
#pragma unroll
    for (int c = 0; c < 3; ++c) U[c * Q3 + q] *= f;
  }
  __syncthreads();
  interp_transpose<T, P>(prm.tab, U, G);
  for (int idx = threadIdx.x; idx < 3 * n3; idx += blockDim.x) {
    bool cons;
    int64_t g = dof_index(prm, P, ex, ey, ez, idx, &cons);
    atomicAdd(&y[g], (double)G[idx]);
  }
}

//-----------------------------------------------------------------------------
// Jacobi diagonal: y += diag(b1 M + K_T) on free DOFs.
// diag_(c,m) = sum_q wdet [ sum_{d,d'} s_d s_d' A_{c d c d'} dN_d dN_d' + b1 rho N^2 ],
// A_{c d c d'} = mu delta_dd' + (c + lambda) H_cd H_cd'.
// With N_m = phi_p(x1) phi_q(x2) phi_r(x3) each product dN_d dN_d' factors
// into 1D tables BB = B.B, BD = B.D, DD = D.D, so seven coefficient fields
// per component are contracted with per-axis product tables.
//-----------------------------------------------------------------------------
template <int P>
constexpr int diag_smem_words() {
  return 7 * (P + 2) * (P + 2) * (P + 2) + 7 * (P + 1) * (P + 2) * (P + 2) + 3 * (P + 2) * (P + 1);
}

template <int P, typename T>
__global__ void __launch_bounds__(elem_threads(P))
diag_kernel(const __grid_constant__ ElemParams<T, P> prm, const T* __restrict__ st, T* __restrict__ y) {
  constexpr int n = P + 1, Q = P + 2, n3 = n * n * n, Q3 = Q * Q * Q;
  // field f: (d, d') pairs then the mass field
  constexpr int fd[7] = {0, 1, 2, 0, 0, 1, -1};
  constexpr int fe[7] = {0, 1, 2, 1, 2, 2, -1};
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* F7 = reinterpret_cast<T*>(smem_raw);      // [7][Q^3], later S1 [7][n][n][Q]
  T* S2 = F7 + 7 * Q3;                         // [7][n][Q][Q]
  T* TB = S2 + 7 * n * Q * Q;                  // BB, BD, DD: [3][Q][n]
  for (int i = threadIdx.x; i < Q * n; i += blockDim.x) {
    const T b = prm.tab.B[i], d = prm.tab.D[i];
    TB[i] = b * b;
    TB[Q * n + i] = b * d;
    TB[2 * Q * n + i] = d * d;
  }
  const int e = blockIdx.x;
  const int ex = e % prm.ne[0], ey = (e / prm.ne[0]) % prm.ne[1], ez = e / (prm.ne[0] * prm.ne[1]);
  const T* ste = st + (int64_t)e * kStateFields * Q3;
  const T sc[3] = {prm.s[0], prm.s[1], prm.s[2]};
  for (int c = 0; c < 3; ++c) {
    __syncthreads();
    for (int q = threadIdx.x; q < Q3; q += blockDim.x) {
      const T wdet = wprod(prm.tab.W, q, Q) * prm.detJ;
      const T a = ste[9 * Q3 + q] + prm.lam;
      const T h[3] = {ste[(c * 3 + 0) * Q3 + q], ste[(c * 3 + 1) * Q3 + q], ste[(c * 3 + 2) * Q3 + q]};
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        const int d = fd[f], d2 = fe[f];
        T v = a * h[d] * h[d2];
        if (d == d2) v += prm.mu;
        else v *= T(2);
        F7[f * Q3 + q] = wdet * sc[d] * sc[d2] * v;
      }
      F7[6 * Q3 + q] = prm.b1 * prm.rho * wdet;
    }
    __syncthreads();
    // axis 2 (z): [f][Q][Q][Q] -> S2 [f][n][Q][Q]
    for (int l = threadIdx.x; l < 7 * Q * Q; l += blockDim.x) {
      const int f = l / (Q * Q), i = l % (Q * Q);
      const int cnt = (fd[f] == 2) + (fe[f] == 2);
      const T* tab = TB + cnt * Q * n;
      T in[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) in[a] = F7[f * Q3 + a * Q * Q + i];
#pragma unroll
      for (int b = 0; b < n; ++b) {
        T acc = T(0);
#pragma unroll
        for (int a = 0; a < Q; ++a) acc += tab[a * n + b] * in[a];
        S2[f * n * Q * Q + b * Q * Q + i] = acc;
      }
    }
    __syncthreads();
    // axis 1 (y): S2 [f][n][Q][Q] -> S1 [f][n][n][Q] (in F7)
    T* S1 = F7;
    for (int l = threadIdx.x; l < 7 * n * Q; l += blockDim.x) {
      const int f = l / (n * Q), rem = l % (n * Q), o = rem / Q, i = rem % Q;
      const int cnt = (fd[f] == 1) + (fe[f] == 1);
      const T* tab = TB + cnt * Q * n;
      T in[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) in[a] = S2[f * n * Q * Q + o * Q * Q + a * Q + i];
#pragma unroll
      for (int b = 0; b < n; ++b) {
        T acc = T(0);
#pragma unroll
        for (int a = 0; a < Q; ++a) acc += tab[a * n + b] * in[a];
        S1[f * n * n * Q + o * n * Q + b * Q + i] = acc;
      }
    }
    __syncthreads();
    // axis 0 (x): sum over fields, one thread per output
    for (int m = threadIdx.x; m < n3; m += blockDim.x) {
      const int p = m % n, rq = m / n;   // rq = r*n + q
      T acc = T(0);
#pragma unroll
      for (int f = 0; f < 7; ++f) {
        const int cnt = (fd[f] == 0) + (fe[f] == 0);
        const T* tab = TB + cnt * Q * n;
#pragma unroll
        for (int a = 0; a < Q; ++a) acc += tab[a * n + p] * S1[f * n * n * Q + rq * Q + a];
      }
      bool cons;
      int64_t g = dof_index(prm, P, ex, ey, ez, c * n3 + m, &cons);
      if (!cons) atomicAdd(&y[g], acc);
    }
  }
}

}  // namespace sdme
