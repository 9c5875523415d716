// Host-side launch wrappers for the element kernels, instantiated once per
// polynomial order in elem_p<P>.cu.
#pragma once

#include "elem_kernels.cuh"
#include "elem_launch.h"

namespace sdme {

// plane-strain quadrilateral launchers (quad_launch.cuh), used for 2D meshes
template <int P>
cudaError_t launch_quad_residual(const HostElemData& h, double b1, const double* u, double* y, double* st64,
                                 float* st32, int* err, cudaStream_t s);
template <int P, typename T, typename TV, bool STIFF>
cudaError_t launch_quad_tangent(const HostElemData& h, double b1, const TV* x, TV* y, const T* st, double* partial,
                                PcgScalars* scal, cudaStream_t s);
template <int P, typename T>
cudaError_t launch_quad_diag(const HostElemData& h, double b1, const T* st, T* y, cudaStream_t s);
template <int P>
cudaError_t launch_quad_mass(const HostElemData& h, const double* x, double* y, cudaStream_t s);
template <int P, typename T>
cudaError_t launch_quad_mass_diag(const HostElemData& h, double b1, T* y, cudaStream_t s);
template <int P>
cudaError_t launch_quad_energy(const HostElemData& h, const double* u, double* partial, unsigned int* counter,
                               double* out, int* err, cudaStream_t s);

template <typename T, int P>
static ElemParams<T, P> make_params(const HostElemData& h, double b1) {
  ElemParams<T, P> p;
  constexpr int n = P + 1, Q = P + 2;
  for (int i = 0; i < Q * n; ++i) {
    p.tab.B[i] = (T)h.B[i];
    p.tab.D[i] = (T)h.D[i];
  }
  for (int i = 0; i < Q; ++i) p.tab.W[i] = (T)h.W[i];
  using E = ElemTables<T, P>;
  for (int i = 0; i < E::QH * E::NE; ++i) p.tab.TE[i] = (T)h.TE[i];
  for (int i = 0; i < E::QH * E::NO; ++i) p.tab.TO[i] = (T)h.TO[i];
  for (int i = 0; i < E::NE; ++i) p.tab.TEm[i] = (T)h.TEm[i];
  for (int i = 0; i < E::QH * E::QH; ++i) {
    p.tab.AH[i] = (T)h.AH[i];
    p.tab.CH[i] = (T)h.CH[i];
  }
  for (int i = 0; i < E::QH; ++i) {
    p.tab.CM[i] = (T)h.CM[i];
    p.tab.DM[i] = (T)h.DM[i];
  }
  for (int q = 0; q < E::QH; ++q) {
    for (int k = 0; k < E::NO; ++k) {
      p.tab.TEO[2 * (q * E::NO + k)] = (T)h.TE[q * E::NE + k];
      p.tab.TEO[2 * (q * E::NO + k) + 1] = (T)h.TO[q * E::NO + k];
    }
    for (int m = 0; m < E::QH; ++m) {
      p.tab.ACH[2 * (q * E::QH + m)] = (T)h.AH[q * E::QH + m];
      p.tab.ACH[2 * (q * E::QH + m) + 1] = (T)h.CH[q * E::QH + m];
    }
  }
  p.pairs = h.pairs;
  p.loc = h.loc;
  for (int d = 0; d < 3; ++d) {
    p.s[d] = (T)h.s[d];
    p.ne[d] = h.ne[d];
    p.N[d] = h.N[d];
  }
  p.detJ = (T)h.detJ;
  p.mu = (T)h.mu;
  p.lam = (T)h.lam;
  p.rho = (T)h.rho;
  p.b1 = (T)b1;
  p.Nn = h.Nn;
  for (int f = 0; f < 6; ++f) p.clamp[f] = h.clamp[f];
  return p;
}

// Opt in to the dynamic shared memory the kernel needs.  Always set: the
// 48 KB default counts static shared memory too (the reduction buffers), so
// a dynamic size just under 48 KB can already fail without it.
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int P>
cudaError_t launch_residual(const HostElemData& h, double b1, const double* u, double* y, double* st64,
                            float* st32, int* err, cudaStream_t s) {
  if (h.dim == 2) return launch_quad_residual<P>(h, b1, u, y, st64, st32, err, s);
  static bool init = false;
  const size_t smem = sizeof(double) * elem_smem_words<P>();
  if (!init) {
    cudaError_t e = set_smem(residual_kernel<P>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<double, P>(h, b1);
  residual_kernel<P><<<h.nelem, elem_threads(P), smem, s>>>(prm, u, y, st64, st32, err);
  return cudaGetLastError();
}

template <int P, typename T, typename TV>
cudaError_t launch_tangent(const HostElemData& h, double b1, const TV* x, TV* y, const T* st,
                           double* partial, PcgScalars* scal, cudaStream_t s, bool defer, int grid, bool pdl) {
  if (h.dim == 2) return launch_quad_tangent<P, T, TV, true>(h, b1, x, y, st, partial, scal, s);
  static bool init = false;
  const size_t smem = sizeof(T) * elem_smem_words<P>();
  if (!init) {
    cudaError_t e = set_smem(tangent_kernel<P, T, TV>, smem);
    if (e == cudaSuccess) e = set_smem(tangent_kernel_strided<P, T, TV>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<T, P>(h, b1);
  if (grid > 0 && grid < h.nelem)
    tangent_kernel_strided<P, T, TV><<<grid, elem_threads(P), smem, s>>>(prm, x, y, st, partial, scal, defer ? 1 : 0,
                                                                         h.nelem);
  else
    return launch_maybe_pdl(tangent_kernel<P, T, TV, true>, dim3(h.nelem), dim3(elem_threads(P)), smem, s, pdl, prm,
                            x, y, st, partial, scal, defer ? 1 : 0);
  return cudaGetLastError();
}

template <int P, typename T, typename TV>
int tangent_resident_ctas() {
  const size_t smem = sizeof(T) * elem_smem_words<P>();
  if (set_smem(tangent_kernel_strided<P, T, TV>, smem) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tangent_kernel_strided<P, T, TV>, elem_threads(P), smem) !=
      cudaSuccess)
    return 0;
  return nb;
}

template <int P, typename T>
cudaError_t launch_diag(const HostElemData& h, double b1, const T* st, T* y, cudaStream_t s) {
  if (h.dim == 2) return launch_quad_diag<P, T>(h, b1, st, y, s);
  static bool init = false;
  const size_t smem = sizeof(T) * diag_smem_words<P>();
  if (!init) {
    cudaError_t e = set_smem(diag_kernel<P, T>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<T, P>(h, b1);
  diag_kernel<P, T><<<h.nelem, elem_threads(P), smem, s>>>(prm, st, y);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_mass(const HostElemData& h, const double* x, double* y, cudaStream_t s) {
  if (h.dim == 2) return launch_quad_mass<P>(h, x, y, s);
  static bool init = false;
  const size_t smem = sizeof(double) * elem_smem_words<P>();
  if (!init) {
    cudaError_t e = set_smem(mass_kernel<P, double>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<double, P>(h, 0.0);
  mass_kernel<P, double><<<h.nelem, elem_threads(P), smem, s>>>(prm, x, y);
  return cudaGetLastError();
}

template <int P, typename T, typename TV>
cudaError_t launch_mass_op(const HostElemData& h, double b1, const TV* x, TV* y, double* partial, PcgScalars* scal,
                           cudaStream_t s, bool defer) {
  if (h.dim == 2) return launch_quad_tangent<P, T, TV, false>(h, b1, x, y, nullptr, partial, scal, s);
  static bool init = false;
  // the mass-only operator never touches the fourth shared field (Gz)
  const size_t smem = sizeof(T) * 9 * Geo<P>::FQ;
  if (!init) {
    cudaError_t e = set_smem(tangent_kernel<P, T, TV, false>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<T, P>(h, b1);
  tangent_kernel<P, T, TV, false><<<h.nelem, elem_threads(P), smem, s>>>(prm, x, y, nullptr, partial, scal,
                                                                          defer ? 1 : 0);
  return cudaGetLastError();
}

template <int P, typename T>
cudaError_t launch_mass_diag(const HostElemData& h, double b1, T* y, cudaStream_t s) {
  if (h.dim == 2) return launch_quad_mass_diag<P, T>(h, b1, y, s);
  auto prm = make_params<T, P>(h, b1);
  mass_diag_kernel<P, T><<<h.nelem, 256, 0, s>>>(prm, y);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_energy(const HostElemData& h, const double* u, double* partial, unsigned int* counter,
                          double* out, int* err, cudaStream_t s) {
  if (h.dim == 2) return launch_quad_energy<P>(h, u, partial, counter, out, err, s);
  static bool init = false;
  const size_t smem = sizeof(double) * elem_smem_words<P>();
  if (!init) {
    cudaError_t e = set_smem(energy_kernel<P>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<double, P>(h, 0.0);
  energy_kernel<P><<<h.nelem, elem_threads(P), smem, s>>>(prm, u, partial, counter, out, err);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_body_load(const HostElemData& h, const double* fq, double* y, cudaStream_t s) {
  if (h.dim == 2) return cudaErrorNotSupported;
  static bool init = false;
  const size_t smem = sizeof(double) * elem_smem_words<P>();
  if (!init) {
    cudaError_t e = set_smem(body_load_kernel<P>, smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  auto prm = make_params<double, P>(h, 0.0);
  body_load_kernel<P><<<h.nelem, elem_threads(P), smem, s>>>(prm, fq, y);
  return cudaGetLastError();
}

#define SDME_INSTANTIATE_ORDER(P)                                                                     \
  template cudaError_t launch_residual<P>(const HostElemData&, double, const double*, double*, double*, \
                                          float*, int*, cudaStream_t);                                \
  template cudaError_t launch_tangent<P, double, double>(const HostElemData&, double, const double*,   \
                                                         double*, const double*, double*, PcgScalars*, \
                                                         cudaStream_t, bool, int, bool);                    \
  template int tangent_resident_ctas<P, double, double>();                                              \
  template cudaError_t launch_tangent<P, float, double>(const HostElemData&, double, const double*,    \
                                                        double*, const float*, double*, PcgScalars*,   \
                                                        cudaStream_t, bool, int, bool);                     \
  template cudaError_t launch_tangent<P, float, float>(const HostElemData&, double, const float*,      \
                                                       float*, const float*, double*, PcgScalars*,     \
                                                       cudaStream_t, bool, int, bool);                      \
  template int tangent_resident_ctas<P, float, float>();                                                \
  template cudaError_t launch_diag<P, double>(const HostElemData&, double, const double*, double*,     \
                                              cudaStream_t);                                          \
  template cudaError_t launch_diag<P, float>(const HostElemData&, double, const float*, float*,        \
                                             cudaStream_t);                                           \
  template cudaError_t launch_mass<P>(const HostElemData&, const double*, double*, cudaStream_t);           \
  template cudaError_t launch_mass_op<P, double, double>(const HostElemData&, double, const double*, double*, \
                                                         double*, PcgScalars*, cudaStream_t, bool);        \
  template cudaError_t launch_mass_op<P, float, float>(const HostElemData&, double, const float*, float*,    \
                                                       double*, PcgScalars*, cudaStream_t, bool);          \
  template cudaError_t launch_mass_diag<P, double>(const HostElemData&, double, double*, cudaStream_t);      \
  template cudaError_t launch_mass_diag<P, float>(const HostElemData&, double, float*, cudaStream_t);        \
  template cudaError_t launch_energy<P>(const HostElemData&, const double*, double*, unsigned int*, double*, \
                                        int*, cudaStream_t);                                                \
  template cudaError_t launch_body_load<P>(const HostElemData&, const double*, double*, cudaStream_t);

}  // namespace sdme
