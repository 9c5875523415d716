// Plane-strain quadrilateral element kernels (tensor products of eq.
// ProdTensorialQuadrado).  One warp per element and kQuadWarps elements per
// CTA: a 2D element has only 2(P+2) lines per stage, so the stages run
// warp-synchronously (__syncwarp) on the warp's own shared-memory slice.
// The 1D machinery (even-odd line contractions, the mirrored-node pairing of
// the nodal basis) is the hexahedral kernels'.
//
// Plane strain: F = [[F_2D, 0], [0, 1]], J = det F_2D, so the in-plane block
// of P = mu (F - F^{-T}) + lambda ln J F^{-T} and of its consistent
// linearisation have the 3D formulas with 2 x 2 matrices.
//
// Per-warp shared memory (T words), four regions of 2 (P+2)((P+2)|1):
//   RU: values / value fluxes U[2][Q][XQ]
//   RX: gathered coefficients X[2][n][XN], then Gx, then the result Y
//   RY: Gy
//   RA: the intermediate A[2][n][XQ] of the x-interpolation (both ways)
// Linearisation state per element: [5][Q^2] = F^{-T} (row major), mu - lambda ln J.
#pragma once

#include "elem_kernels.cuh"

namespace sdme {

constexpr int kQuadWarps = 8;
constexpr int kQuadThreads = 32 * kQuadWarps;
constexpr int kQuadStateFields = 5;

template <int P>
struct QGeo {
  static constexpr int n = P + 1, Q = P + 2;
  static constexpr int XQ = Q | 1, XN = n | 1;
  static constexpr int FQ = Q * XQ;        // one component of a Q x Q field
  static constexpr int REG = 2 * FQ;       // one region
  static constexpr int WORDS = 4 * REG;    // per warp
};

template <int P, typename T>
constexpr size_t quad_smem_bytes() {
  return sizeof(T) * QGeo<P>::WORDS * kQuadWarps;
}

// (c, m) entry of a quad element: global DOF, constrained flag, offset in X.
template <int P, typename T>
__device__ __forceinline__ int64_t quad_entry(const MeshParams<T>& m, int ex, int ey, int idx, bool* cons, int* so) {
  using G = QGeo<P>;
  constexpr int n = P + 1, n2 = n * n;
  const int c = idx / n2, r = idx - c * n2, q = r / n, p = r - q * n;
  const int ix = ex * P + p, iy = ey * P + q;
  *so = c * n * G::XN + q * G::XN + p;
  const unsigned bit = 1u << c;
  *cons = ((ix == 0) && (m.clamp[0] & bit)) || ((ix == m.N[0] - 1) && (m.clamp[1] & bit)) ||
          ((iy == 0) && (m.clamp[2] & bit)) || ((iy == m.N[1] - 1) && (m.clamp[3] & bit));
  return c * m.Nn + (int64_t)iy * m.N[0] + ix;
}

// Forward stages of one element (warp-synchronous): X (RX) -> U (RU) and, if
// GRAD, the reference derivatives Gx (RX), Gy (RY).
template <typename T, int P, bool GRAD>
__device__ __forceinline__ void quad_forward(const ElemTables<T, P>& tb, int pairs, T* sm, int lane) {
  using G = QGeo<P>;
  constexpr int n = G::n, Q = G::Q, XQ = G::XQ, XN = G::XN, FQ = G::FQ;
  T* RU = sm;
  T* RX = sm + G::REG;
  T* RY = sm + 2 * G::REG;
  T* RA = sm + 3 * G::REG;
  for (int l = lane; l < 2 * n; l += 32) {  // x-lines of the coefficients
    const int c = l / n, q = l - c * n;
    T in[n], out[Q];
    load_line(RX + c * n * XN + q * XN, 1, in);
    if (pairs) to_canonical(in);
    eo_interp(tb, in, out);
    store_line(RA + c * n * XQ + q * XQ, 1, out);
  }
  __syncwarp();
  for (int l = lane; l < 2 * Q; l += 32) {  // y-lines at each qx (+ y-derivative)
    const int c = l / Q, qx = l - c * Q;
    T in[n], u[Q];
    load_line(RA + c * n * XQ + qx, XQ, in);
    if (pairs) to_canonical(in);
    eo_interp(tb, in, u);
    store_line(RU + c * FQ + qx, XQ, u);
    if (GRAD) {
      T d[Q];
      eo_deriv(tb, u, d);
      store_line(RY + c * FQ + qx, XQ, d);
    }
  }
  __syncwarp();
  if (GRAD) {
    for (int l = lane; l < 2 * Q; l += 32) {  // x-derivative along each qy row
      const int c = l / Q, qy = l - c * Q;
      T v[Q], d[Q];
      load_line(RU + c * FQ + qy * XQ, 1, v);
      eo_deriv(tb, v, d);
      store_line(RX + c * FQ + qy * XQ, 1, d);
    }
    __syncwarp();
  }
}

// Transposed stages: U (value fluxes) and, if GRAD, Gx, Gy (stress fluxes)
// -> Y (RX, layout of X).
template <typename T, int P, bool GRAD>
__device__ __forceinline__ void quad_transpose(const ElemTables<T, P>& tb, int pairs, T* sm, int lane) {
  using G = QGeo<P>;
  constexpr int n = G::n, Q = G::Q, XQ = G::XQ, XN = G::XN, FQ = G::FQ;
  T* RU = sm;
  T* RX = sm + G::REG;
  T* RY = sm + 2 * G::REG;
  T* RA = sm + 3 * G::REG;
  if (GRAD) {
    for (int l = lane; l < 2 * Q; l += 32) {  // U += DQ^T Gx along x
      const int c = l / Q, qy = l - c * Q;
      T g[Q], r[Q];
      load_line(RX + c * FQ + qy * XQ, 1, g);
      eo_deriv_t(tb, g, r);
      add_line(RU + c * FQ + qy * XQ, 1, r);
    }
    __syncwarp();
  }
  for (int l = lane; l < 2 * Q; l += 32) {  // y: w = U + DQ^T Gy, then B^T w
    const int c = l / Q, qx = l - c * Q;
    T w[Q];
    load_line(RU + c * FQ + qx, XQ, w);
    if (GRAD) {
      T g[Q], r[Q];
      load_line(RY + c * FQ + qx, XQ, g);
      eo_deriv_t(tb, g, r);
#pragma unroll
      for (int a = 0; a < Q; ++a) w[a] += r[a];
    }
    T out[n];
    eo_interp_t(tb, w, out);
    if (pairs) from_canonical(out);
    store_line(RA + c * n * XQ + qx, XQ, out);
  }
  __syncwarp();
  for (int l = lane; l < 2 * n; l += 32) {  // x: B^T
    const int c = l / n, q = l - c * n;
    T in[Q], out[n];
    load_line(RA + c * n * XQ + q * XQ, 1, in);
    eo_interp_t(tb, in, out);
    if (pairs) from_canonical(out);
    store_line(RX + c * n * XN + q * XN, 1, out);
  }
  __syncwarp();
}

// CTA sum of one value per warp in warp order, written to partial[blockIdx.x];
// with a counter, the last CTA (of gridDim.x) sums the partials in order and
// returns true with the total in *total (thread 0); otherwise false.
__device__ __forceinline__ bool quad_cta_reduce(double v, double* partial, unsigned int* counter, double* total) {
  __shared__ double red[kQuadWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kQuadWarps; ++k) s += red[k];
    partial[blockIdx.x] = s;
  }
  if (!counter || !last_arrival(counter, gridDim.x)) return false;
  const double t = ordered_sum(partial, gridDim.x);
  if (threadIdx.x == 0) *total = t;
  return true;
}

// Residual: y += R(u) + b1 M u and the linearisation state at u.
template <int P>
__global__ void __launch_bounds__(kQuadThreads)
quad_residual_kernel(const __grid_constant__ ElemParams<double, P> prm, const double* __restrict__ u,
                     double* __restrict__ y, double* __restrict__ st64, float* __restrict__ st32,
                     int* __restrict__ err) {
  using T = double;
  using G = QGeo<P>;
  constexpr int n = P + 1, Q = P + 2, XQ = G::XQ, FQ = G::FQ, Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * kQuadWarps + w;
  if (e >= prm.ne[0] * prm.ne[1]) return;
  T* sm = reinterpret_cast<T*>(smem_raw) + w * G::WORDS;
  T* RU = sm;
  T* RX = sm + G::REG;
  T* RY = sm + 2 * G::REG;
  const MeshParams<T>& m = prm;
  const int ex = e % m.ne[0], ey = e / m.ne[0];
  for (int idx = lane; idx < 2 * n * n; idx += 32) {
    bool cons;
    int so;
    const int64_t g = quad_entry<P>(m, ex, ey, idx, &cons, &so);
    RX[so] = u[g];
  }
  __syncwarp();
  quad_forward<T, P, true>(prm.tab, prm.pairs, sm, lane);
  for (int q = lane; q < Q2; q += 32) {
    const int qy = q / Q, qx = q - qy * Q;
    const int so = qy * XQ + qx;
    T F[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      F[c][0] = (c == 0 ? T(1) : T(0)) + RX[c * FQ + so] * m.s[0];
      F[c][1] = (c == 1 ? T(1) : T(0)) + RY[c * FQ + so] * m.s[1];
    }
    const T J = F[0][0] * F[1][1] - F[0][1] * F[1][0];
    if (!(J > T(0))) atomicOr(err, 1);
    const T iJ = T(1) / J;
    const T H[2][2] = {{F[1][1] * iJ, -F[1][0] * iJ}, {-F[0][1] * iJ, F[0][0] * iJ}};  // F^{-T}
    const T lnJ = log(J);
    const T a = m.lam * lnJ;
    const T wdet = prm.tab.W[qx] * prm.tab.W[qy] * m.detJ;
    const int64_t o = (int64_t)e * kQuadStateFields * Q2 + q;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const T P0 = m.mu * (F[c][0] - H[c][0]) + a * H[c][0];
      const T P1 = m.mu * (F[c][1] - H[c][1]) + a * H[c][1];
      RX[c * FQ + so] = wdet * P0 * m.s[0];
      RY[c * FQ + so] = wdet * P1 * m.s[1];
      RU[c * FQ + so] *= m.b1 * m.rho * wdet;
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        if (st64) st64[o + (c * 2 + d) * Q2] = H[c][d];
        if (st32) st32[o + (c * 2 + d) * Q2] = (float)H[c][d];
      }
    }
    if (st64) st64[o + 4 * Q2] = m.mu - a;
    if (st32) st32[o + 4 * Q2] = (float)(m.mu - a);
  }
  __syncwarp();
  quad_transpose<T, P, true>(prm.tab, prm.pairs, sm, lane);
  for (int idx = lane; idx < 2 * n * n; idx += 32) {
    bool cons;
    int so;
    const int64_t g = quad_entry<P>(m, ex, ey, idx, &cons, &so);
    atomicAdd(&y[g], RX[so]);
  }
}

// Tangent: y += (b1 M + K_T(u)) x on free DOFs (x taken as 0 on constrained
// ones); with dot_partial / scal, x.(K x) and the PCG step length as in the
// hexahedral kernel.  STIFF = false: the mass-only operator b1 M.
template <int P, typename T, typename TV, bool STIFF>
__global__ void __launch_bounds__(kQuadThreads)
quad_tangent_kernel(const __grid_constant__ ElemParams<T, P> prm, const TV* __restrict__ x, TV* __restrict__ y,
                    const T* __restrict__ st, double* __restrict__ dot_partial, PcgScalars* __restrict__ scal) {
  using G = QGeo<P>;
  constexpr int n = P + 1, Q = P + 2, XQ = G::XQ, FQ = G::FQ, Q2 = Q * Q;
  if (scal && scal->status != 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * kQuadWarps + w;
  const MeshParams<T>& m = prm;
  double dotT = 0.0;
  if (e < m.ne[0] * m.ne[1]) {
    T* sm = reinterpret_cast<T*>(smem_raw) + w * G::WORDS;
    T* RU = sm;
    T* RX = sm + G::REG;
    T* RY = sm + 2 * G::REG;
    const int ex = e % m.ne[0], ey = e / m.ne[0];
    for (int idx = lane; idx < 2 * n * n; idx += 32) {
      bool cons;
      int so;
      const int64_t g = quad_entry<P>(m, ex, ey, idx, &cons, &so);
      RX[so] = cons ? T(0) : (T)x[g];
    }
    __syncwarp();
    quad_forward<T, P, STIFF>(prm.tab, prm.pairs, sm, lane);
    const T* ste = st + (int64_t)e * kQuadStateFields * Q2;
    for (int q = lane; q < Q2; q += 32) {
      const int qy = q / Q, qx = q - qy * Q;
      const int so = qy * XQ + qx;
      const T wdet = prm.tab.W[qx] * prm.tab.W[qy] * m.detJ;
      if constexpr (STIFF) {
        T H[2][2], dF[2][2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
          for (int d = 0; d < 2; ++d) H[c][d] = ste[(c * 2 + d) * Q2 + q];
          dF[c][0] = RX[c * FQ + so] * m.s[0];
          dF[c][1] = RY[c * FQ + so] * m.s[1];
        }
        const T cst = ste[4 * Q2 + q];
        const T tr = H[0][0] * dF[0][0] + H[0][1] * dF[0][1] + H[1][0] * dF[1][0] + H[1][1] * dF[1][1];
        T Wm[2][2];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int j = 0; j < 2; ++j) Wm[a][j] = dF[0][a] * H[0][j] + dF[1][a] * H[1][j];
        const T ltr = m.lam * tr;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const T V0 = H[i][0] * Wm[0][0] + H[i][1] * Wm[1][0];
          const T V1 = H[i][0] * Wm[0][1] + H[i][1] * Wm[1][1];
          RX[i * FQ + so] = wdet * (m.mu * dF[i][0] + cst * V0 + ltr * H[i][0]) * m.s[0];
          RY[i * FQ + so] = wdet * (m.mu * dF[i][1] + cst * V1 + ltr * H[i][1]) * m.s[1];
        }
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) RU[c * FQ + so] *= m.b1 * m.rho * wdet;
    }
    __syncwarp();
    quad_transpose<T, P, STIFF>(prm.tab, prm.pairs, sm, lane);
    for (int idx = lane; idx < 2 * n * n; idx += 32) {
      bool cons;
      int so;
      const int64_t g = quad_entry<P>(m, ex, ey, idx, &cons, &so);
      if (!cons) {
        const T v = RX[so];
        atomicAdd(&y[g], (TV)v);
        if (dot_partial) dotT += (double)(v * (T)x[g]);
      }
    }
  }
  if (dot_partial) {
    double pq = 0.0;
    if (quad_cta_reduce(dotT, dot_partial, scal ? &scal->counter : nullptr, &pq) && scal &&
        threadIdx.x == 0) {
      scal->pq = pq;
      scal->alpha = scal->rz / pq;
      if (!(pq > 0.0) || !isfinite(scal->alpha)) scal->status = kPcgBreakdown;
      scal->counter = 0;
    }
  }
}

// Mass: y += M x (no Dirichlet treatment), float64.
template <int P>
__global__ void __launch_bounds__(kQuadThreads)
quad_mass_kernel(const __grid_constant__ ElemParams<double, P> prm, const double* __restrict__ x,
                 double* __restrict__ y) {
  using T = double;
  using G = QGeo<P>;
  constexpr int n = P + 1, Q = P + 2, XQ = G::XQ, FQ = G::FQ, Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * kQuadWarps + w;
  const MeshParams<T>& m = prm;
  if (e >= m.ne[0] * m.ne[1]) return;
  T* sm = reinterpret_cast<T*>(smem_raw) + w * G::WORDS;
  T* RU = sm;
  T* RX = sm + G::REG;
  const int ex = e % m.ne[0], ey = e / m.ne[0];
  for (int idx = lane; idx < 2 * n * n; idx += 32) {
    bool cons;
    int so;
    const int64_t g = quad_entry<P>(m, ex, ey, idx, &cons, &so);
    RX[so] = x[g];
  }
  __syncwarp();
  quad_forward<T, P, false>(prm.tab, prm.pairs, sm, lane);
  for (int q = lane; q < Q2; q += 32) {
    const int qy = q / Q, qx = q - qy * Q, so = qy * XQ + qx;
    const T f = m.rho * prm.tab.W[qx] * prm.tab.W[qy] * m.detJ;
    RU[so] *= f;
    RU[FQ + so] *= f;
  }
  __syncwarp();
  quad_transpose<T, P, false>(prm.tab, prm.pairs, sm, lane);
  for (int idx = lane; idx < 2 * n * n; idx += 32) {
    bool cons;
    int so;
    const int64_t g = quad_entry<P>(m, ex, ey, idx, &cons, &so);
    atomicAdd(&y[g], RX[so]);
  }
}

// Jacobi diagonal: y += diag(b1 M + K_T) on free DOFs.  Per component, four
// coefficient fields at the Gauss points, (d, d') = (x, x), (y, y), (x, y) and
// the mass field, contracted with the per-axis product tables BB, BD, DD.
template <int P>
__host__ __device__ constexpr size_t quad_diag_words() {
  return (size_t)4 * (P + 2) * (P + 2) + 4 * (P + 1) * (P + 2);  // fields + y-stage results, per warp
}

template <int P, typename T>
__global__ void __launch_bounds__(kQuadThreads)
quad_diag_kernel(const __grid_constant__ ElemParams<T, P> prm, const T* __restrict__ st, T* __restrict__ y) {
  constexpr int n = P + 1, Q = P + 2, Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T TB[3 * Q * n];  // BB, BD, DD [k][Q][n]
  for (int i = threadIdx.x; i < Q * n; i += blockDim.x) {
    const T b = prm.tab.B[i], d = prm.tab.D[i];
    TB[i] = b * b;
    TB[Q * n + i] = b * d;
    TB[2 * Q * n + i] = d * d;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * kQuadWarps + w;
  const MeshParams<T>& m = prm;
  if (e >= m.ne[0] * m.ne[1]) return;
  T* F4 = reinterpret_cast<T*>(smem_raw) + w * quad_diag_words<P>();  // [4][Q2]
  T* S4 = F4 + 4 * Q2;                                                  // [4][n][Q]
  constexpr int cx[4] = {2, 0, 1, 0};  // table index (count of x-derivatives) per field
  constexpr int cy[4] = {0, 2, 1, 0};
  const int ex = e % m.ne[0], ey = e / m.ne[0];
  const T* ste = st + (int64_t)e * kQuadStateFields * Q2;
  for (int c = 0; c < 2; ++c) {
    for (int q = lane; q < Q2; q += 32) {
      const int qy = q / Q, qx = q - qy * Q;
      const T wdet = prm.tab.W[qx] * prm.tab.W[qy] * m.detJ;
      const T a = ste[4 * Q2 + q] + m.lam;
      const T h0 = ste[(c * 2 + 0) * Q2 + q], h1 = ste[(c * 2 + 1) * Q2 + q];
      F4[0 * Q2 + q] = wdet * m.s[0] * m.s[0] * (m.mu + a * h0 * h0);
      F4[1 * Q2 + q] = wdet * m.s[1] * m.s[1] * (m.mu + a * h1 * h1);
      F4[2 * Q2 + q] = wdet * m.s[0] * m.s[1] * T(2) * a * h0 * h1;
      F4[3 * Q2 + q] = m.b1 * m.rho * wdet;
    }
    __syncwarp();
    for (int l = lane; l < 4 * Q; l += 32) {  // y-stage: (field, qx) lines -> n outputs
      const int f = l / Q, qx = l - f * Q;
      const T* tab = TB + cy[f] * Q * n;
      for (int b = 0; b < n; ++b) {
        T acc = T(0);
        for (int qy = 0; qy < Q; ++qy) acc += tab[qy * n + b] * F4[f * Q2 + qy * Q + qx];
        S4[(f * n + b) * Q + qx] = acc;
      }
    }
    __syncwarp();
    for (int o = lane; o < n * n; o += 32) {  // x-stage: outputs (q, p)
      const int qn = o / n, p = o - qn * n;
      T acc = T(0);
      for (int f = 0; f < 4; ++f) {
        const T* tab = TB + cx[f] * Q * n;
        for (int qx = 0; qx < Q; ++qx) acc += tab[qx * n + p] * S4[(f * n + qn) * Q + qx];
      }
      bool cons;
      int so;
      const int64_t g = quad_entry<P>(m, ex, ey, c * n * n + o, &cons, &so);
      if (!cons) atomicAdd(&y[g], acc);
    }
    __syncwarp();
  }
}

// Mass diagonal: y += b1 diag(M) on free DOFs (b1 rho detJ m_p m_q, m_j = sum_k W_k B_kj^2).
template <int P, typename T>
__global__ void __launch_bounds__(kQuadThreads)
quad_mass_diag_kernel(const __grid_constant__ ElemParams<T, P> prm, T* __restrict__ y) {
  constexpr int n = P + 1, Q = P + 2;
  __shared__ T m1[n];
  if (threadIdx.x < n) {
    T acc = T(0);
    for (int k = 0; k < Q; ++k) acc += prm.tab.W[k] * prm.tab.B[k * n + threadIdx.x] * prm.tab.B[k * n + threadIdx.x];
    m1[threadIdx.x] = acc;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * kQuadWarps + w;
  const MeshParams<T>& m = prm;
  if (e >= m.ne[0] * m.ne[1]) return;
  const int ex = e % m.ne[0], ey = e / m.ne[0];
  const T f = m.b1 * m.rho * m.detJ;
  for (int idx = lane; idx < 2 * n * n; idx += 32) {
    bool cons;
    int so;
    const int64_t g = quad_entry<P>(m, ex, ey, idx, &cons, &so);
    const int r = idx % (n * n), q = r / n, p = r - q * n;
    if (!cons) atomicAdd(&y[g], f * m1[p] * m1[q]);
  }
}

// Strain energy (plane strain, eq. hyperelastic strain energy with F_33 = 1):
// the last CTA writes the fixed-order sum to *out.
template <int P>
__global__ void __launch_bounds__(kQuadThreads)
quad_energy_kernel(const __grid_constant__ ElemParams<double, P> prm, const double* __restrict__ u,
                   double* __restrict__ partial, unsigned int* counter, double* out, int* __restrict__ err) {
  using T = double;
  using G = QGeo<P>;
  constexpr int n = P + 1, Q = P + 2, XQ = G::XQ, FQ = G::FQ, Q2 = Q * Q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * kQuadWarps + w;
  const MeshParams<T>& m = prm;
  T acc = T(0);
  if (e < m.ne[0] * m.ne[1]) {
    T* sm = reinterpret_cast<T*>(smem_raw) + w * G::WORDS;
    T* RX = sm + G::REG;
    T* RY = sm + 2 * G::REG;
    const int ex = e % m.ne[0], ey = e / m.ne[0];
    for (int idx = lane; idx < 2 * n * n; idx += 32) {
      bool cons;
      int so;
      const int64_t g = quad_entry<P>(m, ex, ey, idx, &cons, &so);
      RX[so] = u[g];
    }
    __syncwarp();
    quad_forward<T, P, true>(prm.tab, prm.pairs, sm, lane);
    for (int q = lane; q < Q2; q += 32) {
      const int qy = q / Q, qx = q - qy * Q, so = qy * XQ + qx;
      const T F00 = T(1) + RX[so] * m.s[0], F01 = RY[so] * m.s[1];
      const T F10 = RX[FQ + so] * m.s[0], F11 = T(1) + RY[FQ + so] * m.s[1];
      const T J = F00 * F11 - F01 * F10;
      if (!(J > T(0))) atomicOr(err, 1);
      const T lnJ = log(J);
      const T trC = F00 * F00 + F01 * F01 + F10 * F10 + F11 * F11 + T(1);
      acc += prm.tab.W[qx] * prm.tab.W[qy] * m.detJ *
             (T(0.5) * m.mu * (trC - T(3)) - m.mu * lnJ + T(0.5) * m.lam * lnJ * lnJ);
    }
  }
  double tot = 0.0;
  if (quad_cta_reduce(acc, partial, counter, &tot) && threadIdx.x == 0) {
    *out = tot;
    *counter = 0;
  }
}

}  // namespace sdme
