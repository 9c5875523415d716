// Adjoint element kernel (vector-Jacobian product of the internal force) and
// its launcher, instantiated per polynomial order beside the forward kernels.
#pragma once

#include "elem_launch.cuh"

namespace sdme {

//-----------------------------------------------------------------------------
// Adjoint (vector-Jacobian product) of the internal force at u, from the
// linearisation state the residual pass stored (H = F^{-T}, c = mu - lambda ln J):
//   gu += K_T(u) w on every DOF (no Dirichlet treatment: R is defined on all
//         DOFs and its Jacobian K_T is symmetric, so (dR/du)^T w = K_T w);
//   w . dR/dmu     = sum_q w_q detJ (F - F^{-T}) : grad_X w,
//   w . dR/dlambda = sum_q w_q detJ ln J F^{-T} : grad_X w,
// the last two because P = mu (F - F^{-T}) + lambda ln J F^{-T} is linear in
// (mu, lambda).  F = cof(H) / det H and ln J = -ln det H are recovered from
// the state.  Per-element partials go to partial[e] and partial[ne + e]; the
// last CTA sums them in a fixed order into out[0], out[1].
//-----------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(elem_threads(P))
vjp_kernel(const __grid_constant__ ElemParams<double, P> prm, const double* __restrict__ w,
           double* __restrict__ gu, const double* __restrict__ st, double* __restrict__ partial,
           unsigned int* counter, double* __restrict__ out) {
  using T = double;
  using G = Geo<P>;
  constexpr int n = P + 1, Q = P + 2, n3 = n * n * n, Q3 = Q * Q * Q, FQ = G::FQ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* X = sm + 3 * FQ;
  const int e = blockIdx.x;
  const ElemView<ElemParams<double, P>> view(prm, P, e);
  for (int idx = threadIdx.x; idx < 3 * n3; idx += blockDim.x) {
    bool cons;
    int so;
    const int64_t g = entry_index<P>(prm, view, idx, &cons, &so);
    X[so] = w[g];
  }
  __syncthreads();
  forward_stages<T, P, true>(prm.tab, prm.pairs, sm, threadIdx.x);
  const T sc[3] = {prm.s[0], prm.s[1], prm.s[2]};
  const T* ste = st + (int64_t)e * kStateFields * Q3;
  T gmu = T(0), glam = T(0);
  for (int q = threadIdx.x; q < Q3; q += blockDim.x) {
    const int qx = q % Q, qy = (q / Q) % Q, qz = q / (Q * Q);
    const int so = G::pt(qx, qy, qz);
    T H[3][3], dW[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        H[c][d] = ste[(c * 3 + d) * Q3 + q];
        dW[c][d] = sm[(3 + 3 * d + c) * FQ + so] * sc[d];
      }
    const T cst = ste[9 * Q3 + q];
    // F = H^{-T} = cof(H) / det H
    T cof[3][3];
    cof[0][0] = H[1][1] * H[2][2] - H[1][2] * H[2][1];
    cof[0][1] = H[1][2] * H[2][0] - H[1][0] * H[2][2];
    cof[0][2] = H[1][0] * H[2][1] - H[1][1] * H[2][0];
    cof[1][0] = H[0][2] * H[2][1] - H[0][1] * H[2][2];
    cof[1][1] = H[0][0] * H[2][2] - H[0][2] * H[2][0];
    cof[1][2] = H[0][1] * H[2][0] - H[0][0] * H[2][1];
    cof[2][0] = H[0][1] * H[1][2] - H[0][2] * H[1][1];
    cof[2][1] = H[0][2] * H[1][0] - H[0][0] * H[1][2];
    cof[2][2] = H[0][0] * H[1][1] - H[0][1] * H[1][0];
    const T detH = H[0][0] * cof[0][0] + H[0][1] * cof[0][1] + H[0][2] * cof[0][2];
    const T lnJ = -log(detH);
    T tr = T(0), fw = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        tr += H[c][d] * dW[c][d];
        fw += cof[c][d] * dW[c][d];
      }
    const T wdet = prm.tab.W[qx] * prm.tab.W[qy] * prm.tab.W[qz] * prm.detJ;
    gmu += wdet * (fw / detH - tr);
    glam += wdet * lnJ * tr;
    // consistent tangent applied to grad w (as in the tangent kernel)
    T Wm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < 3; ++j) Wm[a][j] = dW[0][a] * H[0][j] + dW[1][a] * H[1][j] + dW[2][a] * H[2][j];
    const T ltr = prm.lam * tr;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const T V = H[i][0] * Wm[0][j] + H[i][1] * Wm[1][j] + H[i][2] * Wm[2][j];
        const T dP = prm.mu * dW[i][j] + cst * V + ltr * H[i][j];
        sm[(3 + 3 * j + i) * FQ + so] = wdet * dP * sc[j];
      }
#pragma unroll
    for (int c = 0; c < 3; ++c) sm[c * FQ + so] = T(0);
  }
  __syncthreads();
  transpose_stages<T, P, true>(prm.tab, prm.pairs, sm, threadIdx.x);
  for (int idx = threadIdx.x; idx < 3 * n3; idx += blockDim.x) {
    bool cons;
    int so;
    const int64_t g = entry_index<P>(prm, view, idx, &cons, &so);
    atomicAdd(&gu[g], X[so]);
  }
  block_sum2(gmu, glam);
  if (threadIdx.x == 0) {
    partial[e] = gmu;
    partial[gridDim.x + e] = glam;
  }
  if (last_block_done(counter)) {
    const double a = ordered_sum(partial, gridDim.x);
    const double b = ordered_sum(partial + gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      out[0] = a;
      out[1] = b;
      *counter = 0;
    }
  }
}

template <int P>
cudaError_t launch_vjp(const HostElemData& h, const double* w, double* gu, const double* st, double* partial,
                       unsigned int* counter, double* out, cudaStream_t s) {
  static bool init = false;
  const size_t smem = sizeof(double) * elem_smem_words<P>();
  if (!init) {
    cudaError_t e = set_smem(vjp_kernel<P>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<double, P>(h, 0.0);
  vjp_kernel<P><<<h.nelem, elem_threads(P), smem, s>>>(prm, w, gu, st, partial, counter, out);
  return cudaGetLastError();
}

#define SDME_INSTANTIATE_ADJOINT(P)                                                                   \
  template cudaError_t launch_vjp<P>(const HostElemData&, const double*, double*, const double*, double*, \
                                     unsigned int*, double*, cudaStream_t);

}  // namespace sdme
