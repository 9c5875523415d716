// Dense element matrices for static condensation: column j of the
// Dirichlet-masked element effective matrix (b1 M + K_T)_e is the tangent
// action on the local unit vector e_j, computed by the same element stages
// as the matrix-free operator (one CTA per (element, column)).
#pragma once

#include "elem_launch.cuh"

namespace sdme {

// Ke[(e * N + j) * N + i] = entry (i, j) of the masked element matrix,
// N = 3 (P+1)^3 in the element's local (component, lattice) order; rows and
// columns of constrained DOFs are zero.
template <int P>
__global__ void __launch_bounds__(elem_threads(P))
cond_columns_kernel(const __grid_constant__ ElemParams<double, P> prm, const double* __restrict__ st,
                    double* __restrict__ Ke) {
  using T = double;
  using G = Geo<P>;
  constexpr int n = P + 1, n3 = n * n * n, N = 3 * n3, FQ = G::FQ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* X = sm + 3 * FQ;
  const int e = blockIdx.x / N, j = blockIdx.x % N;
  const MeshParams<T>& m = prm;
  const ElemView<MeshParams<T>> view(m, P, e);
  bool jcons = false;
  for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
    bool cons;
    int so;
    entry_index<P>(m, view, idx, &cons, &so);
    X[so] = (idx == j && !cons) ? T(1) : T(0);
  }
  {
    bool cons;
    int so;
    entry_index<P>(m, view, j, &cons, &so);
    jcons = cons;
  }
  __syncthreads();
  tangent_core<P, T, true>(prm.tab, prm.pairs, m, e, st, sm, threadIdx.x);
  double* col = Ke + ((int64_t)e * N + j) * N;
  for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
    bool cons;
    int so;
    entry_index<P>(m, view, idx, &cons, &so);
    col[idx] = (cons || jcons) ? 0.0 : X[so];
  }
}

template <int P>
cudaError_t launch_cond_columns(const HostElemData& h, double b1, const double* st, double* Ke, cudaStream_t s) {
  static bool init = false;
  const size_t smem = sizeof(double) * elem_smem_words<P>();
  if (!init) {
    cudaError_t e = set_smem(cond_columns_kernel<P>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  constexpr int N = 3 * (P + 1) * (P + 1) * (P + 1);
  auto prm = make_params<double, P>(h, b1);
  cond_columns_kernel<P><<<(unsigned)((int64_t)h.nelem * N), elem_threads(P), smem, s>>>(prm, st, Ke);
  return cudaGetLastError();
}

#define SDME_INSTANTIATE_COND(P) \
  template cudaError_t launch_cond_columns<P>(const HostElemData&, double, const double*, double*, cudaStream_t);

}  // namespace sdme
