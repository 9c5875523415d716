// Element kernels over a batch of independent meshes of one polynomial
// order: one launch covers up to kBatchLaunchMax problems.  The per-problem
// scalars (MeshParams) and offsets travel in the kernel parameter block next
// to the order's 1D tables, so every CTA finds its problem by a binary
// search over the element prefix and then runs the same element bodies as
// the single-mesh kernels.  Grid: one CTA per element, or a persistent grid
// whose CTAs loop over the elements (chosen per order by the batch's
// launch-configuration tuner).
#pragma once

#include "elem_launch.cuh"

namespace sdme {

constexpr int kBatchLaunchMax = 128;

template <typename T, int P>
struct BatchParams {
  ElemTables<T, P> tab;
  int pairs;
  int nprob;                              // problems in this launch
  int total;                              // elements in this launch
  int estart[kBatchLaunchMax + 1];        // element prefix within the launch
  int pid[kBatchLaunchMax];               // problem index in the batch
  int64_t dof_off[kBatchLaunchMax];       // offset of the problem's vectors
  int64_t st_off[kBatchLaunchMax];        // offset of its Gauss-point state (words)
  int64_t part_off[kBatchLaunchMax];      // offset of its per-element partials
  MeshParams<T> m[kBatchLaunchMax];
  const int* loc[kBatchLaunchMax];        // per-problem offset tables (ElemParams::loc), or null
};
static_assert(sizeof(BatchParams<double, 8>) <= 32000, "batch parameter block exceeds the kernel parameter limit");

template <typename T, int P>
__device__ __forceinline__ int batch_find(const BatchParams<T, P>& bp, int w) {
  int lo = 0, hi = bp.nprob;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (bp.estart[mid] <= w) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <int P>
__global__ void __launch_bounds__(elem_threads(P))
batch_residual_kernel(const __grid_constant__ BatchParams<double, P> bp, const double* __restrict__ u,
                      double* __restrict__ y, double* __restrict__ st64, float* __restrict__ st32,
                      int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  for (int w = blockIdx.x; w < bp.total; w += gridDim.x) {
    const int k = batch_find(bp, w);
    const int64_t off = bp.dof_off[k], so = bp.st_off[k];
    __syncthreads();
    residual_body<P>(bp.tab, bp.pairs, bp.m[k], w - bp.estart[k], u + off, y + off, st64 ? st64 + so : nullptr,
                     st32 ? st32 + so : nullptr, err + bp.pid[k], sm);
  }
}

template <int P, typename T, typename TV>
__global__ void __launch_bounds__(elem_threads(P), tangent_min_blocks<T>())
batch_tangent_kernel(const __grid_constant__ BatchParams<T, P> bp, const TV* __restrict__ x, TV* __restrict__ y,
                     const T* __restrict__ st, double* __restrict__ partial, PcgScalars* __restrict__ scal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  for (int w = blockIdx.x; w < bp.total; w += gridDim.x) {
    const int k = batch_find(bp, w);
    const int64_t off = bp.dof_off[k];
    __syncthreads();
    tangent_body<P, T, TV, true>(bp.tab, bp.pairs, bp.m[k], w - bp.estart[k], x + off, y + off, st + bp.st_off[k],
                                 partial ? partial + bp.part_off[k] : nullptr,
                                 (unsigned)(bp.estart[k + 1] - bp.estart[k]), scal ? scal + bp.pid[k] : nullptr, sm,
                                 bp.loc[k]);
  }
}

template <int P, typename T>
__global__ void __launch_bounds__(elem_threads(P))
batch_diag_kernel(const __grid_constant__ BatchParams<T, P> bp, const T* __restrict__ st, T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  for (int w = blockIdx.x; w < bp.total; w += gridDim.x) {
    const int k = batch_find(bp, w);
    __syncthreads();
    diag_body<P, T>(bp.tab, bp.m[k], w - bp.estart[k], st + bp.st_off[k], y + bp.dof_off[k], sm);
  }
}

template <int P>
__global__ void __launch_bounds__(elem_threads(P))
batch_mass_kernel(const __grid_constant__ BatchParams<double, P> bp, const double* __restrict__ x,
                  double* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  for (int w = blockIdx.x; w < bp.total; w += gridDim.x) {
    const int k = batch_find(bp, w);
    const int64_t off = bp.dof_off[k];
    __syncthreads();
    mass_body<P, double>(bp.tab, bp.pairs, bp.m[k], w - bp.estart[k], x + off, y + off, sm);
  }
}

template <typename T, int P>
static void make_batch_params(const HostElemData& tabs, const HostBatchLaunch& L, double b1, BatchParams<T, P>* bp) {
  const ElemParams<T, P> ep = make_params<T, P>(tabs, b1);
  bp->tab = ep.tab;
  bp->pairs = ep.pairs;
  bp->nprob = (int)L.pid.size();
  bp->total = L.estart.back();
  for (int k = 0; k < bp->nprob; ++k) {
    const HostMesh& h = L.mesh[k];
    MeshParams<T>& m = bp->m[k];
    for (int d = 0; d < 3; ++d) {
      m.s[d] = (T)h.s[d];
      m.ne[d] = h.ne[d];
      m.N[d] = h.N[d];
    }
    m.detJ = (T)h.detJ;
    m.mu = (T)h.mu;
    m.lam = (T)h.lam;
    m.rho = (T)h.rho;
    m.b1 = (T)b1;
    m.Nn = h.Nn;
    for (int f = 0; f < 6; ++f) m.clamp[f] = h.clamp[f];
    bp->estart[k] = L.estart[k];
    bp->pid[k] = L.pid[k];
    bp->dof_off[k] = L.dof_off[k];
    bp->st_off[k] = L.st_off[k];
    bp->part_off[k] = L.part_off[k];
    bp->loc[k] = h.loc;
  }
  bp->estart[bp->nprob] = bp->total;
}

// grid <= 0: one CTA per element; else that many CTAs looping over elements.
static inline unsigned batch_grid(const HostBatchLaunch& L, int grid) {
  const int total = L.estart.back();
  return (unsigned)((grid > 0 && grid < total) ? grid : total);
}

template <int P>
cudaError_t launch_batch_residual(const HostElemData& tabs, const HostBatchLaunch& L, double b1, int grid,
                                  const double* u, double* y, double* st64, float* st32, int* err, cudaStream_t s) {
  static bool init = false;
  const size_t smem = sizeof(double) * elem_smem_words<P>();
  if (!init) {
    cudaError_t e = set_smem(batch_residual_kernel<P>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto* bp = new BatchParams<double, P>;
  make_batch_params<double, P>(tabs, L, b1, bp);
  batch_residual_kernel<P><<<batch_grid(L, grid), elem_threads(P), smem, s>>>(*bp, u, y, st64, st32, err);
  delete bp;
  return cudaGetLastError();
}

template <int P, typename T, typename TV>
cudaError_t launch_batch_tangent(const HostElemData& tabs, const HostBatchLaunch& L, double b1, int grid,
                                 const TV* x, TV* y, const T* st, double* partial, PcgScalars* scal, cudaStream_t s) {
  static bool init = false;
  const size_t smem = sizeof(T) * elem_smem_words<P>();
  if (!init) {
    cudaError_t e = set_smem(batch_tangent_kernel<P, T, TV>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto* bp = new BatchParams<T, P>;
  make_batch_params<T, P>(tabs, L, b1, bp);
  batch_tangent_kernel<P, T, TV><<<batch_grid(L, grid), elem_threads(P), smem, s>>>(*bp, x, y, st, partial, scal);
  delete bp;
  return cudaGetLastError();
}

template <int P, typename T>
cudaError_t launch_batch_diag(const HostElemData& tabs, const HostBatchLaunch& L, double b1, int grid, const T* st,
                              T* y, cudaStream_t s) {
  static bool init = false;
  const size_t smem = sizeof(T) * diag_smem_words<P>();
  if (!init) {
    cudaError_t e = set_smem(batch_diag_kernel<P, T>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto* bp = new BatchParams<T, P>;
  make_batch_params<T, P>(tabs, L, b1, bp);
  batch_diag_kernel<P, T><<<batch_grid(L, grid), elem_threads(P), smem, s>>>(*bp, st, y);
  delete bp;
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_batch_mass(const HostElemData& tabs, const HostBatchLaunch& L, int grid, const double* x,
                              double* y, cudaStream_t s) {
  static bool init = false;
  const size_t smem = sizeof(double) * elem_smem_words<P>();
  if (!init) {
    cudaError_t e = set_smem(batch_mass_kernel<P>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto* bp = new BatchParams<double, P>;
  make_batch_params<double, P>(tabs, L, 0.0, bp);
  batch_mass_kernel<P><<<batch_grid(L, grid), elem_threads(P), smem, s>>>(*bp, x, y);
  delete bp;
  return cudaGetLastError();
}

// Resident CTAs per SM of the batched tangent kernel (0 on error).
template <int P, typename T, typename TV>
int batch_tangent_occupancy() {
  const size_t smem = sizeof(T) * elem_smem_words<P>();
  if (set_smem(batch_tangent_kernel<P, T, TV>, smem) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_tangent_kernel<P, T, TV>, elem_threads(P), smem) !=
      cudaSuccess)
    return 0;
  return nb;
}

#define SDME_INSTANTIATE_BATCH(P)                                                                            \
  template cudaError_t launch_batch_residual<P>(const HostElemData&, const HostBatchLaunch&, double, int,       \
                                                const double*, double*, double*, float*, int*, cudaStream_t);  \
  template cudaError_t launch_batch_tangent<P, double, double>(const HostElemData&, const HostBatchLaunch&,     \
                                                               double, int, const double*, double*,            \
                                                               const double*, double*, PcgScalars*,            \
                                                               cudaStream_t);                                  \
  template cudaError_t launch_batch_tangent<P, float, float>(const HostElemData&, const HostBatchLaunch&,       \
                                                             double, int, const float*, float*, const float*,  \
                                                             double*, PcgScalars*, cudaStream_t);              \
  template cudaError_t launch_batch_tangent<P, float, double>(const HostElemData&, const HostBatchLaunch&,      \
                                                              double, int, const double*, double*,             \
                                                              const float*, double*, PcgScalars*,              \
                                                              cudaStream_t);                                   \
  template int batch_tangent_occupancy<P, float, float>();                                                    \
  template int batch_tangent_occupancy<P, double, double>();                                                  \
  template cudaError_t launch_batch_diag<P, double>(const HostElemData&, const HostBatchLaunch&, double, int,    \
                                                    const double*, double*, cudaStream_t);                     \
  template cudaError_t launch_batch_diag<P, float>(const HostElemData&, const HostBatchLaunch&, double, int,     \
                                                   const float*, float*, cudaStream_t);                        \
  template cudaError_t launch_batch_mass<P>(const HostElemData&, const HostBatchLaunch&, int, const double*,     \
                                            double*, cudaStream_t);

}  // namespace sdme
