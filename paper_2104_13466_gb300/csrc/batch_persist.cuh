// One persistent launch of the batched tangent operator across all order
// groups.  Every CTA has kPersistThreads threads and pulls work items from a
// device counter; an item is up to K_P consecutive elements of one problem
// of order P, processed side by side by K_P groups of G::NT threads (the
// item's "tile"; K_P chosen per order by the batch tuner).  Groups step
// through the element stages together, so the CTA's barriers serve all of
// them; threads outside the groups and groups past the item's element count
// run the stages without touching memory.  Nothing in the kernel waits on
// another CTA: items are claimed with one atomic add each.
#pragma once

#include "elem_kernels.cuh"
#include "elem_launch.h"

namespace sdme {

constexpr int kPersistThreads = 320;   // elem_threads(8): the largest element group

// The 1D tables of every order in one kernel parameter block (the unrolled
// contractions read them as constant-bank operands, as in the per-order
// kernels).
template <typename T>
struct AllTables {
  ElemTables<T, 1> t1;
  ElemTables<T, 2> t2;
  ElemTables<T, 3> t3;
  ElemTables<T, 4> t4;
  ElemTables<T, 5> t5;
  ElemTables<T, 6> t6;
  ElemTables<T, 7> t7;
  ElemTables<T, 8> t8;
  int pairs[9];
  int kper[9];   // elements per item (groups per CTA) for each order
};
static_assert(sizeof(AllTables<double>) <= 30000, "order tables exceed the kernel parameter limit");

template <int P, typename T>
__device__ __forceinline__ const ElemTables<T, P>& tables_of(const AllTables<T>& a) {
  if constexpr (P == 1) return a.t1;
  else if constexpr (P == 2) return a.t2;
  else if constexpr (P == 3) return a.t3;
  else if constexpr (P == 4) return a.t4;
  else if constexpr (P == 5) return a.t5;
  else if constexpr (P == 6) return a.t6;
  else if constexpr (P == 7) return a.t7;
  else return a.t8;
}

// Per-problem data of the persistent launch (device memory).
template <typename T>
struct PersistProb {
  MeshParams<T> m;
  int64_t dof_off, st_off, part_off;
  const int* loc;   // offset table of the tangent gather / scatter, or null
  int pid;          // problem index (PCG scalars)
  int nelem;
};


template <int P, typename T, typename TV>
__device__ __forceinline__ void persist_tile(const ElemTables<T, P>& tb, int pairs, int K, const PersistItem& I,
                                             const PersistProb<T>& pr, const TV* __restrict__ x0,
                                             TV* __restrict__ y0, const T* __restrict__ st0,
                                             double* __restrict__ partial, PcgScalars* __restrict__ scal, T* sm,
                                             double* s_red, int* s_last) {
  using G = Geo<P>;
  constexpr int n = P + 1, n3 = n * n * n, Q = P + 2, Q3 = Q * Q * Q, NT = G::NT;
  constexpr int kOut = 1 << 20;   // thread index of threads outside every group: every loop skips them
  const int g = threadIdx.x / NT;
  const bool member = g < K;
  const int t = member ? (int)threadIdx.x - g * NT : kOut;
  const MeshParams<T>& m = pr.m;
  PcgScalars* sc = scal + pr.pid;
  const bool live = member && g < I.count && *reinterpret_cast<volatile const int*>(&sc->status) == kPcgRunning;
  const int e = I.e0 + (g < I.count ? g : 0);   // groups past the count shadow the first element
  const TV* x = x0 + pr.dof_off;
  TV* y = y0 + pr.dof_off;
  const T* st = st0 + pr.st_off;
  T* smg = sm + (member ? g : 0) * G::WORDS;
  T* X = smg + 3 * G::FQ;
  const ElemView<MeshParams<T>> view(m, P, e);
  const bool fast = (G::XN == n) && pr.loc != nullptr && !view.boundary;
  if (live) {
    if (t == 0) prefetch_l2(st + (int64_t)e * kStateFields * Q3, sizeof(T) * kStateFields * Q3);
    if (fast) {
      const TV* xb = x + view.base;
      for (int idx = t; idx < 3 * n3; idx += NT) X[idx] = (T)xb[__ldg(pr.loc + idx)];
    } else {
      for (int idx = t; idx < 3 * n3; idx += NT) {
        bool cons;
        int so;
        const int64_t gi = entry_index<P>(m, view, idx, &cons, &so);
        X[so] = cons ? T(0) : (T)x[gi];
      }
    }
  } else if (member) {
    // a group without an element (or of a converged problem) computes on zeros
    for (int idx = t; idx < 3 * n3; idx += NT) {
      bool cons;
      int so;
      entry_index<P>(m, view, idx, &cons, &so);
      X[so] = T(0);
    }
  }
  __syncthreads();
  double dotT = tangent_core<P, T, true>(tb, pairs, m, e, st, smg, t);
  constexpr bool RELOAD = sizeof(T) == 8;  // float64: x_e . y_e from a second read of x
  if (live) {
    if (fast) {
      const TV* xb = x + view.base;
      TV* yb = y + view.base;
      for (int idx = t; idx < 3 * n3; idx += NT) {
        const int o = __ldg(pr.loc + idx);
        const T v = X[idx];
        atomicAdd(&yb[o], (TV)v);
        if (RELOAD) dotT += (double)(v * (T)xb[o]);
      }
    } else {
      for (int idx = t; idx < 3 * n3; idx += NT) {
        bool cons;
        int so;
        const int64_t gi = entry_index<P>(m, view, idx, &cons, &so);
        if (!cons) {
          const T v = X[so];
          atomicAdd(&y[gi], (TV)v);
          if (RELOAD) dotT += (double)(v * (T)x[gi]);
        }
      }
    }
  }
  // x_e . (K_e x_e) per group: warp sums (groups are whole warps), then the
  // group's warps in order; the problem's last element to arrive sums the
  // problem's partials (one warp, fixed order) into the step length
  if (!live) dotT = 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dotT += __shfl_xor_sync(0xffffffffu, dotT, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = dotT;
  __syncthreads();
  if (member && t == 0) {
    int last = 0;
    if (live) {
      double tot = 0.0;
      for (int w = 0; w < NT / 32; ++w) tot += s_red[g * (NT / 32) + w];
      partial[pr.part_off + e] = tot;
      __threadfence();
      last = atomicAdd(&sc->counter, 1u) == (unsigned)(pr.nelem - 1);
    }
    s_last[g] = last;
  }
  __syncthreads();
  if (member && s_last[g] && t < 32) {
    __threadfence();
    double s = 0.0;
    for (int i = t; i < pr.nelem; i += 32) s += __ldcg(partial + pr.part_off + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (t == 0) {
      sc->pq = s;
      sc->alpha = sc->rz / s;
      if (!(s > 0.0) || !isfinite(sc->alpha)) sc->status = kPcgBreakdown;
      sc->counter = 0;
    }
  }
}

template <typename T, typename TV>
__global__ void __launch_bounds__(kPersistThreads, tangent_min_blocks<T>())
batch_tangent_persistent(const __grid_constant__ AllTables<T> at, const PersistItem* __restrict__ items,
                         const int* __restrict__ nitems, int* __restrict__ queue,
                         const PersistProb<T>* __restrict__ probs, const TV* __restrict__ x, TV* __restrict__ y,
                         const T* __restrict__ st, double* __restrict__ partial, PcgScalars* __restrict__ scal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ int s_item;
  __shared__ double s_red[kPersistThreads / 32];
  __shared__ int s_last[kPersistThreads / 32];
  const int n_items = *nitems;
  for (;;) {
    __syncthreads();   // everyone has read the previous s_item
    if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const PersistItem I = items[it];
    const PersistProb<T>& pr = probs[I.prob];
    switch (I.P) {
#define SDME_PERSIST_CASE(PP)                                                                                    \
  case PP:                                                                                                       \
    persist_tile<PP, T, TV>(tables_of<PP>(at), at.pairs[PP], at.kper[PP], I, pr, x, y, st, partial, scal, sm, \
                            s_red, s_last);                                                                      \
    break;
      SDME_PERSIST_CASE(1)
      SDME_PERSIST_CASE(2)
      SDME_PERSIST_CASE(3)
      SDME_PERSIST_CASE(4)
      SDME_PERSIST_CASE(5)
      SDME_PERSIST_CASE(6)
      SDME_PERSIST_CASE(7)
      SDME_PERSIST_CASE(8)
#undef SDME_PERSIST_CASE
      default:
        break;
    }
  }
}

}  // namespace sdme
