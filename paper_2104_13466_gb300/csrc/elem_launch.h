// Declarations of the per-order element-kernel launchers (no device code).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace sdme {

struct PcgScalars;

// Everything an element kernel needs, in float64 on the host; each launcher
// converts it into its kernel-parameter block.
struct HostElemData {
  int P = 0;
  int dim = 3;                       // 3: hexahedra; 2: plane-strain quadrilaterals (ne[2] = N[2] = 1)
  int nelem = 0;
  std::vector<double> B, D, DQ, W;   // Q x n, Q x n, Q x Q, Q (lattice order)
  // even-odd half tables (eo_tables.h) and the nodal-pairing flag
  std::vector<double> TE, TO, TEm, AH, CH, CM, DM;
  int pairs = 0;
  double s[3] = {0, 0, 0};           // 2 / h_d
  double detJ = 0;
  double mu = 0, lam = 0, rho = 0;
  int ne[3] = {0, 0, 0};
  int N[3] = {0, 0, 0};
  int64_t Nn = 0;
  unsigned clamp[6] = {0, 0, 0, 0, 0, 0};
  const int* loc = nullptr;          // device offset table of the tangent gather / scatter (or null)
};

// Per-problem scalars of a batched launch (float64 on the host).
struct HostMesh {
  double s[3] = {0, 0, 0};
  double detJ = 0, mu = 0, lam = 0, rho = 0;
  int ne[3] = {0, 0, 0};
  int N[3] = {0, 0, 0};
  int64_t Nn = 0;
  unsigned clamp[6] = {0, 0, 0, 0, 0, 0};
  const int* loc = nullptr;          // device offset table of the tangent gather / scatter (or null)
};

// One batched element launch: up to kBatchLaunchMax problems of one order.
struct HostBatchLaunch {
  std::vector<int> estart;                  // element prefix, size nprob + 1
  std::vector<int> pid;                     // problem index in the batch
  std::vector<int64_t> dof_off, st_off, part_off;
  std::vector<HostMesh> mesh;
};

template <int P>
cudaError_t launch_batch_residual(const HostElemData& tabs, const HostBatchLaunch& L, double b1, int grid,
                                  const double* u, double* y, double* st64, float* st32, int* err, cudaStream_t s);
template <int P, typename T, typename TV>
cudaError_t launch_batch_tangent(const HostElemData& tabs, const HostBatchLaunch& L, double b1, int grid,
                                 const TV* x, TV* y, const T* st, double* partial, PcgScalars* scal, cudaStream_t s);
template <int P, typename T, typename TV>
int batch_tangent_occupancy();
template <int P, typename T>
cudaError_t launch_batch_diag(const HostElemData& tabs, const HostBatchLaunch& L, double b1, int grid, const T* st,
                              T* y, cudaStream_t s);
template <int P>
cudaError_t launch_batch_mass(const HostElemData& tabs, const HostBatchLaunch& L, int grid, const double* x,
                              double* y, cudaStream_t s);

// Cross-order persistent launch of the batched tangent (batch_persist.cuh).
// An item is up to kper[P] consecutive elements e0 .. e0 + count - 1 of the
// problem with index `prob` in the per-problem table, of order P.
struct PersistItem {
  int P, prob, e0, count;
};

struct HostPersist {
  const HostElemData* tabs[9] = {};   // the 1D tables of each order present (else null)
  int kper[9] = {};                   // elements per item for each order
};

// One problem of the per-problem table (built on the host, uploaded as is).
struct HostPersistProb {
  HostMesh mesh;
  int64_t dof_off = 0, st_off = 0, part_off = 0;
  int pid = 0, nelem = 0;
};

// Bytes of one device-side table entry, and the host image of the table
// (b1 is the mass coefficient of the operator).
template <typename T>
size_t persist_prob_bytes();
template <typename T>
void persist_probs_image(const std::vector<HostPersistProb>& probs, double b1, std::vector<unsigned char>& out);
// Dynamic shared memory of the launch and its resident CTAs per SM (0 on error).
template <typename T>
size_t persist_smem(const HostPersist& hp);
template <typename T, typename TV>
int persist_occupancy(const HostPersist& hp);
template <typename T, typename TV>
cudaError_t launch_batch_persistent(const HostPersist& hp, int grid, const PersistItem* items, const int* nitems,
                                    int* queue, const void* probs, const TV* x, TV* y, const T* st,
                                    double* partial, PcgScalars* scal, cudaStream_t s);
constexpr int kPersistMaxTile = 4;    // elements per item considered by the tuner

template <int P>
cudaError_t launch_cond_columns(const HostElemData& h, double b1, const double* st, double* Ke, cudaStream_t s);

template <int P>
cudaError_t launch_residual(const HostElemData& h, double b1, const double* u, double* y, double* st64,
                            float* st32, int* err, cudaStream_t s);
// grid > 0 (and below the element count): that many CTAs, each serving every
// grid-th element, with one step-length partial per CTA; else one CTA per element.
// pdl: launch as the programmatic dependent of the previous kernel in the
// stream (one CTA per element only).
template <int P, typename T, typename TV>
cudaError_t launch_tangent(const HostElemData& h, double b1, const TV* x, TV* y, const T* st,
                           double* partial, PcgScalars* scal, cudaStream_t s, bool defer = false, int grid = 0,
                           bool pdl = false);

// Kernel launch, optionally as the programmatic dependent of the previous
// kernel in the stream (the kernel then calls pdl_wait() before it reads
// anything that kernel writes).
template <typename... KArgs, typename... Args>
cudaError_t launch_maybe_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                             Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
// Resident CTAs per SM of the fixed-grid tangent kernel (0 on error).
template <int P, typename T, typename TV>
int tangent_resident_ctas();
template <int P, typename T>
cudaError_t launch_diag(const HostElemData& h, double b1, const T* st, T* y, cudaStream_t s);
template <int P>
cudaError_t launch_mass(const HostElemData& h, const double* x, double* y, cudaStream_t s);
template <int P, typename T, typename TV>
cudaError_t launch_mass_op(const HostElemData& h, double b1, const TV* x, TV* y, double* partial, PcgScalars* scal,
                           cudaStream_t s, bool defer = false);
template <int P, typename T>
cudaError_t launch_mass_diag(const HostElemData& h, double b1, T* y, cudaStream_t s);
template <int P>
cudaError_t launch_body_load(const HostElemData& h, const double* fq, double* y, cudaStream_t s);
template <int P>
cudaError_t launch_vjp(const HostElemData& h, const double* w, double* gu, const double* st, double* partial,
                       unsigned int* counter, double* out, cudaStream_t s);
template <int P>
cudaError_t launch_energy(const HostElemData& h, const double* u, double* partial, unsigned int* counter,
                          double* out, int* err, cudaStream_t s);

}  // namespace sdme
