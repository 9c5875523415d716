// Launchers of the plane-strain quadrilateral kernels (one warp per element,
// kQuadWarps elements per CTA); the element launchers of elem_launch.cuh
// forward here for two-dimensional meshes.
#pragma once

#include "elem_launch.cuh"
#include "quad_kernels.cuh"

namespace sdme {

inline unsigned quad_grid(const HostElemData& h) { return (unsigned)((h.nelem + kQuadWarps - 1) / kQuadWarps); }

template <int P>
cudaError_t launch_quad_residual(const HostElemData& h, double b1, const double* u, double* y, double* st64,
                                 float* st32, int* err, cudaStream_t s) {
  static bool init = false;
  const size_t smem = quad_smem_bytes<P, double>();
  if (!init) {
    cudaError_t e = set_smem(quad_residual_kernel<P>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<double, P>(h, b1);
  quad_residual_kernel<P><<<quad_grid(h), kQuadThreads, smem, s>>>(prm, u, y, st64, st32, err);
  return cudaGetLastError();
}

template <int P, typename T, typename TV, bool STIFF>
cudaError_t launch_quad_tangent(const HostElemData& h, double b1, const TV* x, TV* y, const T* st, double* partial,
                                PcgScalars* scal, cudaStream_t s) {
  static bool init = false;
  const size_t smem = quad_smem_bytes<P, T>();
  if (!init) {
    cudaError_t e = set_smem(quad_tangent_kernel<P, T, TV, STIFF>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<T, P>(h, b1);
  quad_tangent_kernel<P, T, TV, STIFF><<<quad_grid(h), kQuadThreads, smem, s>>>(prm, x, y, st, partial, scal);
  return cudaGetLastError();
}

template <int P, typename T>
cudaError_t launch_quad_diag(const HostElemData& h, double b1, const T* st, T* y, cudaStream_t s) {
  static bool init = false;
  const size_t smem = sizeof(T) * quad_diag_words<P>() * kQuadWarps;
  if (!init) {
    cudaError_t e = set_smem(quad_diag_kernel<P, T>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<T, P>(h, b1);
  quad_diag_kernel<P, T><<<quad_grid(h), kQuadThreads, smem, s>>>(prm, st, y);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_quad_mass(const HostElemData& h, const double* x, double* y, cudaStream_t s) {
  static bool init = false;
  const size_t smem = quad_smem_bytes<P, double>();
  if (!init) {
    cudaError_t e = set_smem(quad_mass_kernel<P>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<double, P>(h, 0.0);
  quad_mass_kernel<P><<<quad_grid(h), kQuadThreads, smem, s>>>(prm, x, y);
  return cudaGetLastError();
}

template <int P, typename T>
cudaError_t launch_quad_mass_diag(const HostElemData& h, double b1, T* y, cudaStream_t s) {
  auto prm = make_params<T, P>(h, b1);
  quad_mass_diag_kernel<P, T><<<quad_grid(h), kQuadThreads, 0, s>>>(prm, y);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_quad_energy(const HostElemData& h, const double* u, double* partial, unsigned int* counter,
                               double* out, int* err, cudaStream_t s) {
  static bool init = false;
  const size_t smem = quad_smem_bytes<P, double>();
  if (!init) {
    cudaError_t e = set_smem(quad_energy_kernel<P>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<double, P>(h, 0.0);
  quad_energy_kernel<P><<<quad_grid(h), kQuadThreads, smem, s>>>(prm, u, partial, counter, out, err);
  return cudaGetLastError();
}

}  // namespace sdme
