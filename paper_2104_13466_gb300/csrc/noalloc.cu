// Allocation-free variant of the tangent matvec, for callers that cannot
// call cudaMalloc (see sdme_tangent_apply_noalloc in include/sdme.h).
//
// The linearisation state at u and the internal-force vector that the
// linearisation pass produces as a by-product live in one file-scope device
// array of fixed size instead of in a context.  The entry point builds its
// kernel parameter block on the stack from the caller's 1D tables, so it
// performs no host or device allocation.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/sdme.h"
#include "elem_kernels.cuh"
#include "eo_tables.h"

using namespace sdme;

namespace {

// 2^21 float64 words = 16 MiB, held by every GPU that loads the library.
constexpr size_t kScratchWords = size_t(1) << 21;
// Words reserved at the start of the array: word 0 holds the error flag.
constexpr size_t kHeaderWords = 32;

static __device__ __align__(256) double g_noalloc_scratch[kScratchWords];

// y = x on constrained DOFs, 0 elsewhere (start of the masked apply).
__global__ void __launch_bounds__(256) noalloc_mask_init(MeshInfo mi, const double* __restrict__ x,
                                                         double* __restrict__ y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < mi.ndof;
       g += (int64_t)gridDim.x * blockDim.x)
    y[g] = dof_constrained(mi, g) ? x[g] : 0.0;
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device; the first call
// per device queries it (cudaGetSymbolAddress) and caches it.
cudaError_t scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

// Derivative of the Lagrange polynomials through the Q Gauss points at each
// Gauss point (barycentric weights; fixed-size arrays, no allocation).
template <int Q>
void gauss_derivative_matrix(const double* xq, double* DQ) {
  double wb[Q];
  for (int j = 0; j < Q; ++j) {
    wb[j] = 1.0;
    for (int k = 0; k < Q; ++k)
      if (k != j) wb[j] /= (xq[j] - xq[k]);
  }
  for (int q = 0; q < Q; ++q) {
    double diag = 0.0;
    for (int m = 0; m < Q; ++m) {
      if (m == q) continue;
      const double v = (wb[m] / wb[q]) / (xq[q] - xq[m]);
      DQ[q * Q + m] = v;
      diag -= v;
    }
    DQ[q * Q + q] = diag;
  }
}

template <int P>
sdme_status run(const sdme_mesh_desc* mesh, const sdme_material* mat, const double* xq, const double* wq,
                const double* B, const double* D, const double* u, double b1, const double* x, double* y,
                cudaStream_t s) {
  constexpr int n = P + 1, Q = P + 2, Q3 = Q * Q * Q;
  ElemParams<double, P> prm;
  for (int i = 0; i < Q * n; ++i) {
    prm.tab.B[i] = B[i];
    prm.tab.D[i] = D[i];
  }
  for (int q = 0; q < Q; ++q) prm.tab.W[q] = wq[q];
  double DQ[Q * Q];
  gauss_derivative_matrix<Q>(xq, DQ);
  const int sym = build_eo_tables(P, B, DQ, prm.tab.TE, prm.tab.TO, prm.tab.TEm, prm.tab.AH, prm.tab.CH, prm.tab.CM,
                                  prm.tab.DM);
  if (sym == kEoNone) return SDME_EUNSUPPORTED;
  prm.pairs = sym == kEoNodalPairs ? 1 : 0;
  double h[3];
  int64_t N[3];
  for (int d = 0; d < 3; ++d) {
    h[d] = mesh->length[d] / mesh->nelem[d];
    prm.s[d] = 2.0 / h[d];
    prm.ne[d] = mesh->nelem[d];
    N[d] = (int64_t)mesh->nelem[d] * P + 1;
    prm.N[d] = (int)N[d];
  }
  // sizes bounded in floating point first (no integer overflow for any mesh)
  if (3.0 * (double)N[0] * (double)N[1] * (double)N[2] +
          (double)mesh->nelem[0] * mesh->nelem[1] * mesh->nelem[2] * kStateFields * Q3 >
      (double)(kScratchWords - kHeaderWords))
    return SDME_EINVAL;
  prm.detJ = h[0] * h[1] * h[2] / 8.0;
  prm.mu = mat->mu;
  prm.lam = mat->lambda;
  prm.rho = mat->rho;
  prm.b1 = 0.0;
  prm.Nn = N[0] * N[1] * N[2];
  for (int f = 0; f < 6; ++f) prm.clamp[f] = mesh->clamp[f] & 7u;
  const int64_t nelem = (int64_t)mesh->nelem[0] * mesh->nelem[1] * mesh->nelem[2];
  const int64_t ndof = 3 * prm.Nn;
  const int64_t state_words = nelem * kStateFields * Q3;
  if ((uint64_t)(kHeaderWords + ndof + state_words) > kScratchWords) return SDME_EINVAL;

  double* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return SDME_ECUDA;
  int* err = reinterpret_cast<int*>(base);
  double* R = base + kHeaderWords;            // discarded internal force
  double* st = R + ndof;                      // linearisation state at u
  // the error flag and the atomically accumulated R must start at zero
  if (cudaMemsetAsync(base, 0, sizeof(double) * (kHeaderWords + ndof), s) != cudaSuccess) return SDME_ECUDA;

  const int threads = elem_threads(P);
  const size_t smem = sizeof(double) * elem_smem_words<P>();
  if (cudaFuncSetAttribute(residual_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(tangent_kernel<P, double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return SDME_ECUDA;
  residual_kernel<P><<<(unsigned)nelem, threads, smem, s>>>(prm, u, R, st, nullptr, err);
  MeshInfo mi;
  for (int d = 0; d < 3; ++d) mi.N[d] = prm.N[d];
  mi.Nn = prm.Nn;
  mi.ndof = ndof;
  for (int f = 0; f < 6; ++f) mi.clamp[f] = prm.clamp[f];
  noalloc_mask_init<<<152 * 4, 256, 0, s>>>(mi, x, y);
  prm.b1 = b1;
  tangent_kernel<P, double, double><<<(unsigned)nelem, threads, smem, s>>>(prm, x, y, st, nullptr, nullptr);
  if (cudaGetLastError() != cudaSuccess) return SDME_ECUDA;
  int err_h = 0;
  if (cudaMemcpyAsync(&err_h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SDME_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SDME_ECUDA;
  return err_h ? SDME_NONPOSITIVE_J : SDME_OK;
}

}  // namespace

extern "C" sdme_status sdme_tangent_apply_noalloc(const sdme_mesh_desc* mesh, const sdme_material* mat, int P,
                                                  const double* xq, const double* wq, const double* B,
                                                  const double* D, const double* u_dev, double b1,
                                                  const double* x_dev, double* y_dev, void* stream) {
  if (!mesh || !mat || !xq || !wq || !B || !D || !u_dev || !x_dev || !y_dev) return SDME_EINVAL;
  // hexahedral meshes only (nelem[2] = 0, a plane-strain mesh, is rejected here)
  for (int d = 0; d < 3; ++d)
    if (mesh->nelem[d] < 1 || mesh->nelem[d] > (1 << 24) || !(mesh->length[d] > 0.0) ||
        !std::isfinite(mesh->length[d]))
      return SDME_EINVAL;
  if (!(mat->mu > 0.0) || !(mat->lambda >= 0.0) || !(mat->rho >= 0.0) || !std::isfinite(mat->mu) ||
      !std::isfinite(mat->lambda) || !std::isfinite(mat->rho))
    return SDME_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  switch (P) {
    case 1: return run<1>(mesh, mat, xq, wq, B, D, u_dev, b1, x_dev, y_dev, s);
    case 2: return run<2>(mesh, mat, xq, wq, B, D, u_dev, b1, x_dev, y_dev, s);
    case 3: return run<3>(mesh, mat, xq, wq, B, D, u_dev, b1, x_dev, y_dev, s);
    case 4: return run<4>(mesh, mat, xq, wq, B, D, u_dev, b1, x_dev, y_dev, s);
    case 5: return run<5>(mesh, mat, xq, wq, B, D, u_dev, b1, x_dev, y_dev, s);
    case 6: return run<6>(mesh, mat, xq, wq, B, D, u_dev, b1, x_dev, y_dev, s);
    case 7: return run<7>(mesh, mat, xq, wq, B, D, u_dev, b1, x_dev, y_dev, s);
    case 8: return run<8>(mesh, mat, xq, wq, B, D, u_dev, b1, x_dev, y_dev, s);
    default: return SDME_EINVAL;
  }
}
