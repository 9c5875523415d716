// Host side of the cross-order persistent batched tangent launch: the
// parameter block with every order's tables, the per-problem table image,
// occupancy and the launch.  Instantiated for float32 and float64 operators.
#include <algorithm>
#include <cstring>

#include "batch_persist.cuh"
#include "elem_launch.cuh"

namespace sdme {

namespace {

template <typename T, int P>
void fill_order(const HostPersist& hp, ElemTables<T, P>& dst, AllTables<T>* at) {
  if (!hp.tabs[P]) return;
  const ElemParams<T, P> ep = make_params<T, P>(*hp.tabs[P], 0.0);
  dst = ep.tab;
  at->pairs[P] = ep.pairs;
}

template <typename T>
void fill_tables(const HostPersist& hp, AllTables<T>* at) {
  fill_order<T, 1>(hp, at->t1, at);
  fill_order<T, 2>(hp, at->t2, at);
  fill_order<T, 3>(hp, at->t3, at);
  fill_order<T, 4>(hp, at->t4, at);
  fill_order<T, 5>(hp, at->t5, at);
  fill_order<T, 6>(hp, at->t6, at);
  fill_order<T, 7>(hp, at->t7, at);
  fill_order<T, 8>(hp, at->t8, at);
  for (int P = 0; P <= 8; ++P) at->kper[P] = hp.kper[P];
}

constexpr int kWords[9] = {0,
                           Geo<1>::WORDS,
                           Geo<2>::WORDS,
                           Geo<3>::WORDS,
                           Geo<4>::WORDS,
                           Geo<5>::WORDS,
                           Geo<6>::WORDS,
                           Geo<7>::WORDS,
                           Geo<8>::WORDS};

}  // namespace

template <typename T>
size_t persist_prob_bytes() {
  return sizeof(PersistProb<T>);
}

template <typename T>
void persist_probs_image(const std::vector<HostPersistProb>& probs, double b1, std::vector<unsigned char>& out) {
  out.assign(probs.size() * sizeof(PersistProb<T>), 0);
  for (size_t i = 0; i < probs.size(); ++i) {
    const HostPersistProb& h = probs[i];
    PersistProb<T> pp{};
    for (int d = 0; d < 3; ++d) {
      pp.m.s[d] = (T)h.mesh.s[d];
      pp.m.ne[d] = h.mesh.ne[d];
      pp.m.N[d] = h.mesh.N[d];
    }
    pp.m.detJ = (T)h.mesh.detJ;
    pp.m.mu = (T)h.mesh.mu;
    pp.m.lam = (T)h.mesh.lam;
    pp.m.rho = (T)h.mesh.rho;
    pp.m.b1 = (T)b1;
    pp.m.Nn = h.mesh.Nn;
    for (int f = 0; f < 6; ++f) pp.m.clamp[f] = h.mesh.clamp[f];
    pp.dof_off = h.dof_off;
    pp.st_off = h.st_off;
    pp.part_off = h.part_off;
    pp.loc = h.mesh.loc;
    pp.pid = h.pid;
    pp.nelem = h.nelem;
    std::memcpy(out.data() + i * sizeof(PersistProb<T>), &pp, sizeof(pp));
  }
}

template <typename T>
size_t persist_smem(const HostPersist& hp) {
  size_t words = 0;
  for (int P = 1; P <= 8; ++P)
    if (hp.tabs[P]) words = std::max(words, (size_t)std::max(1, hp.kper[P]) * kWords[P]);
  return sizeof(T) * words;
}

template <typename T, typename TV>
int persist_occupancy(const HostPersist& hp) {
  const size_t smem = persist_smem<T>(hp);
  if (set_smem(batch_tangent_persistent<T, TV>, smem) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_tangent_persistent<T, TV>, kPersistThreads, smem) !=
      cudaSuccess)
    return 0;
  return nb;
}

template <typename T, typename TV>
cudaError_t launch_batch_persistent(const HostPersist& hp, int grid, const PersistItem* items, const int* nitems,
                                    int* queue, const void* probs, const TV* x, TV* y, const T* st,
                                    double* partial, PcgScalars* scal, cudaStream_t s) {
  for (int P = 1; P <= 8; ++P) {
    const int nt = (3 * (P + 2) * (P + 2) + 31) / 32 * 32;   // Geo<P>::NT
    if (hp.tabs[P] && (hp.kper[P] < 1 || hp.kper[P] * nt > kPersistThreads)) return cudaErrorInvalidValue;
  }
  const size_t smem = persist_smem<T>(hp);
  cudaError_t e = set_smem(batch_tangent_persistent<T, TV>, smem);
  if (e != cudaSuccess) return e;
  auto* at = new AllTables<T>();
  fill_tables<T>(hp, at);
  batch_tangent_persistent<T, TV><<<grid, kPersistThreads, smem, s>>>(
      *at, items, nitems, queue, reinterpret_cast<const PersistProb<T>*>(probs), x, y, st, partial, scal);
  delete at;
  return cudaGetLastError();
}

template size_t persist_prob_bytes<float>();
template size_t persist_prob_bytes<double>();
template void persist_probs_image<float>(const std::vector<HostPersistProb>&, double, std::vector<unsigned char>&);
template void persist_probs_image<double>(const std::vector<HostPersistProb>&, double, std::vector<unsigned char>&);
template size_t persist_smem<float>(const HostPersist&);
template size_t persist_smem<double>(const HostPersist&);
template int persist_occupancy<float, float>(const HostPersist&);
template int persist_occupancy<double, double>(const HostPersist&);
template cudaError_t launch_batch_persistent<float, float>(const HostPersist&, int, const PersistItem*, const int*,
                                                           int*, const void*, const float*, float*, const float*,
                                                           double*, PcgScalars*, cudaStream_t);
template cudaError_t launch_batch_persistent<double, double>(const HostPersist&, int, const PersistItem*, const int*,
                                                             int*, const void*, const double*, double*,
                                                             const double*, double*, PcgScalars*, cudaStream_t);

}  // namespace sdme
