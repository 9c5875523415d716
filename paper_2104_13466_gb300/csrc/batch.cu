// Batched solves over many independent box meshes (host side of the
// sdme_batch_* entry points).  Problems are grouped by polynomial order;
// every element operation is one launch per group (up to 128 problems per
// launch), every per-DOF operation one launch for the whole batch, and the
// PCG iterations of all problems run as one captured CUDA graph per chunk.
// The PCG operator can instead run as one persistent launch across all
// order groups (batch_persist.cuh), with the elements per work item chosen
// per order by the tuner; the tuner keeps whichever form is faster.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/sdme.h"
#include "basis1d.h"
#include "batch_vec.cuh"
#include "elem_launch.h"
#include "eo_tables.h"

using namespace sdme;

namespace {

constexpr int kLaunchMax = 128;        // problems per element launch (kBatchLaunchMax)
constexpr int kChunk = 16;             // PCG iterations per captured graph
constexpr int64_t kSegAlign = 8;       // segment alignment in vector entries (64 B in float64)
constexpr int kVecGridTotal = 152 * 8; // per-DOF grid of the batch-wide (unsplit) kernels

struct Prob {
  sdme_problem d{};
  int P = 0, Q = 0;
  int64_t nelem = 0, ndof = 0, off = 0, st_off = 0, part_off = 0;
  HostMesh hm;
  MeshInfo mi{};
  int group = 0;
};

struct Group {
  int P = 0;
  HostElemData tabs;
  std::vector<int> probs;
  std::vector<HostBatchLaunch> launches;
  std::vector<HostBatchLaunch> run_launches;  // launches restricted to the problems whose PCG is running
  int64_t nelem = 0;
  int grid = 0;      // 0: one CTA per element; else persistent CTAs
  float tuned_ms = 0.f;
};

template <typename F>
cudaError_t dispatch_order(int P, F&& f) {
  switch (P) {
    case 1: return f(std::integral_constant<int, 1>());
    case 2: return f(std::integral_constant<int, 2>());
    case 3: return f(std::integral_constant<int, 3>());
    case 4: return f(std::integral_constant<int, 4>());
    case 5: return f(std::integral_constant<int, 5>());
    case 6: return f(std::integral_constant<int, 6>());
    case 7: return f(std::integral_constant<int, 7>());
    case 8: return f(std::integral_constant<int, 8>());
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

}  // namespace

struct sdme_batch {
  int nprob = 0;
  sdme_precision prec = SDME_FP64;
  sdme_basis_desc basis{};
  cudaStream_t stream = nullptr;
  cudaError_t last_cuda = cudaSuccess;
  std::vector<Prob> probs;
  std::vector<Group> groups;
  int64_t total = 0, nelem_total = 0, st_total = 0;
  int vec_grid = 0;
  // device
  BatchVecInfo* info = nullptr;
  int* cta_prob = nullptr;
  int* active = nullptr;
  int* err = nullptr;
  PcgScalars* scal = nullptr;
  double* partial = nullptr;
  unsigned int* dcount = nullptr;
  double* dnorm = nullptr;
  double* st64 = nullptr;
  float* st32 = nullptr;
  double *r64 = nullptr, *p64 = nullptr, *q64 = nullptr, *d64 = nullptr, *x64 = nullptr;
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr, *x32 = nullptr;
  double *un = nullptr, *ahat = nullptr, *mhat = nullptr, *y = nullptr, *psi = nullptr, *du = nullptr;
  int* loc = nullptr;         // per-problem tangent offset tables (even orders), concatenated
  // pinned host mirrors
  PcgScalars* scal_h = nullptr;
  double* dnorm_h = nullptr;
  int* err_h = nullptr;
  int* active_h = nullptr;
  // PCG chunk graph on a private stream
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double gb1 = 0.0;
  int gsize = 0;
  std::vector<int> grun;      // running problems the captured chunk was built for
  bool warm = false;          // kernels' attributes set (first chunk ran directly)
  int64_t launches = 0;
  // cross-order persistent PCG operator
  int persist_mode = -1;      // -1: the tuner decides, 0: per-order launches, 1: persistent
  bool persist_on = false;
  bool persist_use = false;   // the current chunk graph uses the persistent launch (>= 2 running orders)
  float persist_order_ms[9] = {-1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f, -1.f};   // tuner, per order
  int kper[9] = {0, 1, 1, 1, 1, 1, 1, 1, 1};
  float persist_ms = -1.f, groups_ms = -1.f;
  int persist_grid = 0;       // resident CTAs of the persistent launch
  int persist_items_n = 0;    // work items uploaded (the launch needs no more CTAs than that)
  int persist_run_orders[9] = {};   // orders among the uploaded items (they set the launch's shared memory)
  double persist_b1 = -1.0;   // b1 of the uploaded per-problem table
  PersistItem* items = nullptr;
  int* nitems = nullptr;
  PersistItem* items_h = nullptr;   // pinned staging of the item list (its count follows the items)
  int persist_grid_cache[512] = {}; // resident-CTA grid per set of running orders (bit P-1 per order)
  int* queue = nullptr;
  unsigned char* pprobs = nullptr;
};

#define B_CUDA(call)                 \
  do {                               \
    cudaError_t e_ = (call);         \
    if (e_ != cudaSuccess) {         \
      b->last_cuda = e_;             \
      return SDME_ECUDA;             \
    }                                \
  } while (0)

#define B_TRY(call)               \
  do {                            \
    sdme_status s_ = (call);      \
    if (s_ != SDME_OK) return s_; \
  } while (0)

namespace {

void batch_free(sdme_batch* b) {
  void* dev[] = {b->items, b->nitems, b->queue, b->pprobs,
                 b->info, b->cta_prob, b->active, b->err, b->scal, b->partial, b->dcount, b->dnorm,
                 b->st64, b->st32, b->r64, b->p64, b->q64, b->d64, b->x64, b->r32, b->p32, b->q32,
                 b->d32, b->x32, b->un, b->ahat, b->mhat, b->y, b->psi, b->du, b->loc};
  for (void* p : dev)
    if (p) cudaFree(p);
  void* host[] = {b->scal_h, b->dnorm_h, b->err_h, b->active_h, b->items_h};
  for (void* p : host)
    if (p) cudaFreeHost(p);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->side) cudaStreamDestroy(b->side);
}

// 1D tables of one order (same construction as a context's).
bool build_group_tables(const sdme_basis_desc* basis, int P, HostElemData& h, int* sym) {
  Basis1D bs;
  if (!bs.build(P, (int)basis->kind, basis->k, basis->lambda, basis->start_nodal != 0, basis->jacobi_alpha,
                basis->jacobi_beta))
    return false;
  const int n = P + 1, Q = P + 2;
  h.P = P;
  h.B.resize(Q * n);
  h.D.resize(Q * n);
  h.DQ.resize(Q * Q);
  h.W.resize(Q);
  std::vector<double> xq(Q);
  gauss_legendre(Q, xq.data(), h.W.data());
  bs.tables(Q, xq.data(), h.B.data(), h.D.data());
  collocation_derivative(Q, xq.data(), h.DQ.data());
  const EoSizes z(P);
  h.TE.resize(z.QH * z.NE);
  h.TO.resize(z.QH * z.NO);
  h.TEm.resize(z.NE);
  h.AH.resize(z.QH * z.QH);
  h.CH.resize(z.QH * z.QH);
  h.CM.resize(z.QH);
  h.DM.resize(z.QH);
  *sym = build_eo_tables(P, h.B.data(), h.DQ.data(), h.TE.data(), h.TO.data(), h.TEm.data(), h.AH.data(),
                         h.CH.data(), h.CM.data(), h.DM.data());
  h.pairs = *sym == kEoNodalPairs ? 1 : 0;
  return true;
}

sdme_status b_check_err(sdme_batch* b) {
  B_CUDA(cudaMemcpyAsync(b->err_h, b->err, sizeof(int) * b->nprob, cudaMemcpyDeviceToHost, b->stream));
  B_CUDA(cudaStreamSynchronize(b->stream));
  bool bad = false;
  for (int i = 0; i < b->nprob; ++i) bad = bad || b->err_h[i] != 0;
  if (bad) {
    B_CUDA(cudaMemsetAsync(b->err, 0, sizeof(int) * b->nprob, b->stream));
    return SDME_NONPOSITIVE_J;
  }
  return SDME_OK;
}

sdme_status b_residual(sdme_batch* b, double b1, const double* u, double* y) {
  B_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * b->total, b->stream));
  float* st32 = b->prec == SDME_MIXED_FP32 ? b->st32 : nullptr;
  for (Group& g : b->groups)
    for (const HostBatchLaunch& L : g.launches) {
      B_CUDA(dispatch_order(g.P, [&](auto Pc) {
        return launch_batch_residual<decltype(Pc)::value>(g.tabs, L, b1, g.grid, u, y, b->st64, st32, b->err,
                                                          b->stream);
      }));
      b->launches += 1;
    }
  return SDME_OK;
}

template <typename T>
const T* b_state(sdme_batch* b) {
  if constexpr (sizeof(T) == 8) return b->st64;
  else return b->st32;
}

// The persistent launch's view of the batch: the tables and tile of each
// order among the uploaded work items (the launch's shared memory and
// resident CTAs follow from those orders only).
HostPersist b_persist_desc(sdme_batch* b) {
  HostPersist hp;
  for (Group& g : b->groups) {
    if (!b->persist_run_orders[g.P]) continue;
    hp.tabs[g.P] = &g.tabs;
    hp.kper[g.P] = b->kper[g.P];
  }
  return hp;
}

// Uploads the work items for the problems in `run` (all when null), largest
// order first, kper[P] consecutive elements per item, and the per-problem
// table when b1 changed.  Stream-ordered on the batch's stream.
sdme_status b_persist_items(sdme_batch* b, const std::vector<int>* run, double b1, int only_P = 0) {
  std::vector<int> order;
  if (run) order = *run;
  else
    for (int i = 0; i < b->nprob; ++i) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->probs[a].P > b->probs[c].P; });
  std::vector<PersistItem> items;
  for (int i : order) {
    const Prob& pr = b->probs[i];
    if (only_P && pr.P != only_P) continue;
    const int K = std::max(1, b->kper[pr.P]);
    for (int64_t e = 0; e < pr.nelem; e += K)
      items.push_back(PersistItem{pr.P, i, (int)e, (int)std::min<int64_t>(K, pr.nelem - e)});
  }
  const int n = (int)items.size();
  b->persist_items_n = n;
  for (int P = 0; P <= 8; ++P) b->persist_run_orders[P] = 0;
  for (const PersistItem& it : items) b->persist_run_orders[it.P] = 1;
  // staged in pinned memory (the caller reads the PCG status, a
  // synchronisation, before it stages the next list), count after the items
  std::memcpy(b->items_h, items.data(), sizeof(PersistItem) * n);
  std::memcpy(reinterpret_cast<int*>(b->items_h + n), &n, sizeof(int));
  B_CUDA(cudaMemsetAsync(b->queue, 0, sizeof(int), b->stream));
  if (n > 0)
    B_CUDA(cudaMemcpyAsync(b->items, b->items_h, sizeof(PersistItem) * n, cudaMemcpyHostToDevice, b->stream));
  B_CUDA(cudaMemcpyAsync(b->nitems, b->items_h + n, sizeof(int), cudaMemcpyHostToDevice, b->stream));
  if (b->persist_b1 != b1) {
    std::vector<HostPersistProb> hp(b->nprob);
    for (int i = 0; i < b->nprob; ++i) {
      const Prob& pr = b->probs[i];
      hp[i].mesh = pr.hm;
      hp[i].dof_off = pr.off;
      hp[i].st_off = pr.st_off;
      hp[i].part_off = pr.part_off;
      hp[i].pid = i;
      hp[i].nelem = (int)pr.nelem;
    }
    std::vector<unsigned char> img;
    if (b->prec == SDME_MIXED_FP32) persist_probs_image<float>(hp, b1, img);
    else persist_probs_image<double>(hp, b1, img);
    B_CUDA(cudaMemcpyAsync(b->pprobs, img.data(), img.size(), cudaMemcpyHostToDevice, b->stream));
    b->persist_b1 = b1;
    // the pageable table must stay valid until its copy has run
    B_CUDA(cudaStreamSynchronize(b->stream));
  }
  return SDME_OK;
}

// reset_queue: clear the work counter first (else the preceding PCG update
// kernel has cleared it, or the item upload did)
template <typename T, typename TV>
sdme_status b_persist_launch(sdme_batch* b, const TV* x, TV* y, double* partial, PcgScalars* scal,
                             bool reset_queue = false) {
  if (reset_queue) B_CUDA(cudaMemsetAsync(b->queue, 0, sizeof(int), b->stream));
  const HostPersist hp = b_persist_desc(b);
  const int grid = std::max(1, std::min(b->persist_grid, b->persist_items_n));
  B_CUDA((launch_batch_persistent<T, TV>(hp, grid, b->items, b->nitems, b->queue, b->pprobs, x, y,
                                          b_state<T>(b), partial, scal, b->stream)));
  b->launches += 1;
  return SDME_OK;
}

sdme_status b_persist_grid(sdme_batch* b) {
  int mask = 0;
  for (int P = 1; P <= 8; ++P) mask |= b->persist_run_orders[P] ? (1 << (P - 1)) : 0;
  if (b->persist_grid_cache[mask] > 0) {
    b->persist_grid = b->persist_grid_cache[mask];
    return SDME_OK;
  }
  const HostPersist hp = b_persist_desc(b);
  const int occ = b->prec == SDME_MIXED_FP32 ? persist_occupancy<float, float>(hp)
                                             : persist_occupancy<double, double>(hp);
  int dev = 0, sms = 0;
  B_CUDA(cudaGetDevice(&dev));
  B_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (occ < 1) return SDME_ECUDA;
  b->persist_grid = occ * sms;
  b->persist_grid_cache[mask] = b->persist_grid;
  return SDME_OK;
}

template <typename T, typename TV>
sdme_status b_tangent_group(sdme_batch* b, Group& g, double b1, int grid, const TV* x, TV* y, double* partial,
                            PcgScalars* scal, bool running_only = false) {
  for (const HostBatchLaunch& L : running_only ? g.run_launches : g.launches) {
    B_CUDA(dispatch_order(g.P, [&](auto Pc) {
      return launch_batch_tangent<decltype(Pc)::value, T, TV>(g.tabs, L, b1, grid, x, y, b_state<T>(b), partial,
                                                              scal, b->stream);
    }));
    b->launches += 1;
  }
  return SDME_OK;
}

template <typename T, typename TV>
sdme_status b_tangent(sdme_batch* b, double b1, const TV* x, TV* y, double* partial, PcgScalars* scal,
                      bool running_only = false) {
  for (Group& g : b->groups)
    B_TRY((b_tangent_group<T, TV>(b, g, b1, g.grid, x, y, partial, scal, running_only)));
  return SDME_OK;
}

// Element launches of every group restricted to the problems in `run`
// (sorted), so that converged problems cost no CTAs in later iterations.
void build_run_launches(sdme_batch* b, const std::vector<int>& run) {
  std::vector<char> on(b->nprob, 0);
  for (int i : run) on[i] = 1;
  for (Group& g : b->groups) {
    g.run_launches.clear();
    for (const HostBatchLaunch& L : g.launches) {
      HostBatchLaunch R;
      int acc = 0;
      for (size_t k = 0; k < L.pid.size(); ++k) {
        if (!on[L.pid[k]]) continue;
        R.estart.push_back(acc);
        R.pid.push_back(L.pid[k]);
        R.dof_off.push_back(L.dof_off[k]);
        R.st_off.push_back(L.st_off[k]);
        R.part_off.push_back(L.part_off[k]);
        R.mesh.push_back(L.mesh[k]);
        acc += L.estart[k + 1] - L.estart[k];
      }
      if (R.pid.empty()) continue;
      R.estart.push_back(acc);
      g.run_launches.push_back(R);
    }
  }
}

template <typename T>
sdme_status b_diag(sdme_batch* b, double b1, T* d) {
  B_CUDA(cudaMemsetAsync(d, 0, sizeof(T) * b->total, b->stream));
  for (Group& g : b->groups)
    for (const HostBatchLaunch& L : g.launches) {
      B_CUDA(dispatch_order(g.P, [&](auto Pc) {
        return launch_batch_diag<decltype(Pc)::value, T>(g.tabs, L, b1, g.grid, b_state<T>(b), d, b->stream);
      }));
      b->launches += 1;
    }
  kb_diag_finish<T><<<b->vec_grid, kVecThreads, 0, b->stream>>>(b->info, b->cta_prob, d, 1);
  B_CUDA(cudaGetLastError());
  b->launches += 1;
  return SDME_OK;
}

sdme_status b_mass(sdme_batch* b, const double* x, double* y) {
  B_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * b->total, b->stream));
  for (Group& g : b->groups)
    for (const HostBatchLaunch& L : g.launches) {
      B_CUDA(dispatch_order(g.P, [&](auto Pc) {
        return launch_batch_mass<decltype(Pc)::value>(g.tabs, L, g.grid, x, y, b->stream);
      }));
      b->launches += 1;
    }
  return SDME_OK;
}

// Runs on the private stream: it waits for the caller's stream on entry and
// the caller's stream waits for it on exit.
struct BatchSideScope {
  sdme_batch* b;
  cudaStream_t user;
  explicit BatchSideScope(sdme_batch* bb) : b(bb), user(bb->stream) {
    cudaEventRecord(b->ev_fork, user);
    cudaStreamWaitEvent(b->side, b->ev_fork, 0);
    b->stream = b->side;
  }
  ~BatchSideScope() {
    cudaEventRecord(b->ev_join, b->side);
    cudaStreamWaitEvent(user, b->ev_join, 0);
    b->stream = user;
  }
};

template <typename T, typename TV>
sdme_status b_pcg_chunk(sdme_batch* b, double b1, TV* r, TV* p, TV* q, TV* dinv, TV* xv) {
  for (int j = 0; j < kChunk; ++j) {
    if (b->persist_use) B_TRY((b_persist_launch<T, TV>(b, p, q, b->partial, b->scal)));
    else B_TRY((b_tangent<T, TV>(b, b1, p, q, b->partial, b->scal, true)));
    kb_pcg_update<TV><<<b->vec_grid, kVecThreads, 0, b->stream>>>(b->info, b->cta_prob, xv, r, p, q, dinv, b->scal,
                                                                  b->partial, b->persist_use ? b->queue : nullptr);
    kb_pcg_direction<TV><<<b->vec_grid, kVecThreads, 0, b->stream>>>(b->info, b->cta_prob, r, dinv, p, b->scal);
    b->launches += 2;
  }
  B_CUDA(cudaGetLastError());
  return SDME_OK;
}

// Jacobi PCG on (b1 M + K_T) for every problem with active[p] != 0 (the
// others get x = 0).  rhs, x_out: float64 concatenated vectors.
template <typename T, typename TV>
sdme_status b_pcg(sdme_batch* b, double b1, const double* rhs, double* x_out, double rtol, int maxit, TV* r, TV* p,
                  TV* q, TV* dinv, TV* xv) {
  BatchSideScope scope(b);
  B_TRY(b_diag<T>(b, b1, (T*)dinv));
  kb_pcg_init<TV><<<b->vec_grid, kVecThreads, 0, b->stream>>>(b->info, b->cta_prob, rhs, dinv, xv, r, p, q,
                                                              b->scal, b->partial, b->active, rtol, maxit);
  B_CUDA(cudaGetLastError());
  b->launches += 1;
  auto read_status = [&](std::vector<int>& run) -> sdme_status {
    B_CUDA(cudaMemcpyAsync(b->scal_h, b->scal, sizeof(PcgScalars) * b->nprob, cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(cudaStreamSynchronize(b->stream));
    run.clear();
    for (int i = 0; i < b->nprob; ++i)
      if (b->scal_h[i].status == kPcgRunning) run.push_back(i);
    return SDME_OK;
  };
  std::vector<int> run;
  B_TRY(read_status(run));
  while (!run.empty()) {
    // the captured chunk covers the running problems only; it is rebuilt
    // whenever that set (or the operator) changes.  Launch accounting: one
    // executed chunk = kChunk x (element launches + update + direction).
    const int64_t l0 = b->launches;
    if (!b->gexec || run != b->grun || b->gb1 != b1 || b->gsize != (int)sizeof(T)) {
      if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
      }
      build_run_launches(b, run);
      // the persistent launch merges orders; with one order running the
      // per-order launch is that order's single launch (and measured faster)
      int orders_running = 0;
      {
        bool seen[9] = {};
        for (int i : run) seen[b->probs[i].P] = true;
        for (int P = 1; P <= 8; ++P) orders_running += seen[P] ? 1 : 0;
      }
      b->persist_use = b->persist_on && (orders_running >= 2 || b->persist_mode == 1);
      if (b->persist_use) {
        B_TRY(b_persist_items(b, &run, b1));
        B_TRY(b_persist_grid(b));
      }
      if (!b->warm) {  // the first chunk runs directly (sets the kernels' attributes)
        B_TRY((b_pcg_chunk<T, TV>(b, b1, r, p, q, dinv, xv)));
        b->warm = true;
        B_TRY(read_status(run));
        continue;
      }
      const int64_t lc = b->launches;
      cudaGraph_t g = nullptr;
      B_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      sdme_status cs = b_pcg_chunk<T, TV>(b, b1, r, p, q, dinv, xv);
      cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
      if (cs != SDME_OK) return cs;
      B_CUDA(ce);
      ce = cudaGraphInstantiate(&b->gexec, g, 0);
      cudaGraphDestroy(g);
      B_CUDA(ce);
      b->gb1 = b1;
      b->gsize = (int)sizeof(T);
      b->grun = run;
      b->launches = lc;  // captured, not executed
    }
    B_CUDA(cudaGraphLaunch(b->gexec, b->stream));
    int64_t per = 2 * kChunk;
    if (b->persist_use) per += kChunk;
    else
      for (const Group& g : b->groups) per += kChunk * (int64_t)g.run_launches.size();
    b->launches = l0 + per;
    B_TRY(read_status(run));
  }
  k_to_double<TV><<<kVecGridTotal, kVecThreads, 0, b->stream>>>(b->total, xv, 1.0, x_out);
  B_CUDA(cudaGetLastError());
  b->launches += 1;
  return SDME_OK;
}

sdme_status b_pcg_dispatch(sdme_batch* b, double b1, const double* rhs, double* x, double rtol, int maxit) {
  if (b->prec == SDME_MIXED_FP32)
    return b_pcg<float, float>(b, b1, rhs, x, rtol, maxit, b->r32, b->p32, b->q32, b->d32, b->x32);
  return b_pcg<double, double>(b, b1, rhs, x, rtol, maxit, b->r64, b->p64, b->q64, b->d64, b->x64);
}

}  // namespace

extern "C" {

sdme_status sdme_batch_create(sdme_batch** out, const sdme_problem* probs, int nprob, const sdme_basis_desc* basis,
                              sdme_precision prec, void* cuda_stream) {
  if (!out || !probs || nprob < 1 || !basis) return SDME_EINVAL;
  *out = nullptr;
  if (prec != SDME_FP64 && prec != SDME_MIXED_FP32) return SDME_EINVAL;
  if (basis->kind < SDME_NODAL || basis->kind > SDME_NODAL_LUMPED) return SDME_EINVAL;
  if (basis->kind == SDME_NODAL_LUMPED) return SDME_EUNSUPPORTED;  // the batched step uses the consistent mass
  if (basis->kind >= SDME_SDME_M && (basis->k < 0.0 || basis->k > 1.0)) return SDME_EINVAL;
  for (int i = 0; i < nprob; ++i) {
    const sdme_problem& d = probs[i];
    if (d.P < 1 || d.P > kMaxP) return SDME_EINVAL;
    for (int k = 0; k < 3; ++k)
      if (d.mesh.nelem[k] < 1 || !(d.mesh.length[k] > 0.0)) return SDME_EINVAL;
    if (!(d.mat.mu > 0.0) || !(d.mat.lambda >= 0.0) || !(d.mat.rho >= 0.0)) return SDME_EINVAL;
    const int64_t ne = (int64_t)d.mesh.nelem[0] * d.mesh.nelem[1] * d.mesh.nelem[2];
    if (ne > 0x7fffffff / 2) return SDME_EINVAL;
  }
  sdme_batch* b = new (std::nothrow) sdme_batch();
  if (!b) return SDME_ENOMEM;
  b->nprob = nprob;
  b->prec = prec;
  b->basis = *basis;
  b->stream = (cudaStream_t)cuda_stream;
  b->probs.resize(nprob);
  // order groups
  for (int i = 0; i < nprob; ++i) {
    Prob& pr = b->probs[i];
    pr.d = probs[i];
    pr.P = probs[i].P;
    pr.Q = pr.P + 2;
    int gi = -1;
    for (size_t k = 0; k < b->groups.size(); ++k)
      if (b->groups[k].P == pr.P) gi = (int)k;
    if (gi < 0) {
      Group g;
      g.P = pr.P;
      int sym = kEoNone;
      if (!build_group_tables(basis, pr.P, g.tabs, &sym)) {
        delete b;
        return SDME_EINVAL;
      }
      if (sym == kEoNone) {
        delete b;
        return SDME_EUNSUPPORTED;
      }
      b->groups.push_back(g);
      gi = (int)b->groups.size() - 1;
    }
    pr.group = gi;
    b->groups[gi].probs.push_back(i);
  }
  // layout: vectors, state, element partials; per-DOF CTA split
  std::vector<BatchVecInfo> info(nprob);
  std::vector<int> cta_prob;
  for (int i = 0; i < nprob; ++i) {
    Prob& pr = b->probs[i];
    const sdme_mesh_desc& m = pr.d.mesh;
    const int P = pr.P, Q = pr.Q;
    pr.nelem = (int64_t)m.nelem[0] * m.nelem[1] * m.nelem[2];
    int64_t N[3];
    for (int d = 0; d < 3; ++d) {
      N[d] = (int64_t)m.nelem[d] * P + 1;
      const double h = m.length[d] / m.nelem[d];
      pr.hm.s[d] = 2.0 / h;
      pr.hm.ne[d] = m.nelem[d];
      pr.hm.N[d] = (int)N[d];
      pr.mi.N[d] = (int)N[d];
    }
    pr.hm.detJ = (m.length[0] / m.nelem[0]) * (m.length[1] / m.nelem[1]) * (m.length[2] / m.nelem[2]) / 8.0;
    pr.hm.mu = pr.d.mat.mu;
    pr.hm.lam = pr.d.mat.lambda;
    pr.hm.rho = pr.d.mat.rho;
    pr.hm.Nn = N[0] * N[1] * N[2];
    for (int f = 0; f < 6; ++f) pr.hm.clamp[f] = pr.mi.clamp[f] = m.clamp[f] & 7u;
    pr.mi.Nn = pr.hm.Nn;
    pr.ndof = 3 * pr.hm.Nn;
    pr.mi.ndof = pr.ndof;
    pr.off = b->total;
    b->total += (pr.ndof + kSegAlign - 1) / kSegAlign * kSegAlign;
    pr.st_off = b->st_total;
    b->st_total += pr.nelem * kStateFields * (int64_t)Q * Q * Q;
    pr.part_off = b->nelem_total;
    b->nelem_total += pr.nelem;
    const int ncta = (int)std::max<int64_t>(1, std::min<int64_t>((pr.ndof + 2047) / 2048, 152 * 4));
    info[i].mi = pr.mi;
    info[i].off = pr.off;
    info[i].cta0 = (int)cta_prob.size();
    info[i].ncta = ncta;
    for (int c = 0; c < ncta; ++c) cta_prob.push_back(i);
  }
  b->vec_grid = (int)cta_prob.size();
  for (Group& g : b->groups) {
    for (size_t s0 = 0; s0 < g.probs.size(); s0 += kLaunchMax) {
      HostBatchLaunch L;
      int acc = 0;
      for (size_t k = s0; k < std::min(g.probs.size(), s0 + kLaunchMax); ++k) {
        const Prob& pr = b->probs[g.probs[k]];
        L.estart.push_back(acc);
        L.pid.push_back(g.probs[k]);
        L.dof_off.push_back(pr.off);
        L.st_off.push_back(pr.st_off);
        L.part_off.push_back(pr.part_off);
        L.mesh.push_back(pr.hm);
        acc += (int)pr.nelem;
      }
      L.estart.push_back(acc);
      g.nelem += acc;
      g.launches.push_back(L);
    }
  }
  const size_t nt = (size_t)b->total, np = (size_t)nprob;
  const size_t npart = (size_t)std::max<int64_t>(b->nelem_total, 2 * (int64_t)b->vec_grid) + 64;
  bool ok = dalloc(&b->info, np) == cudaSuccess && dalloc(&b->cta_prob, cta_prob.size()) == cudaSuccess &&
            dalloc(&b->active, np) == cudaSuccess && dalloc(&b->err, np) == cudaSuccess &&
            dalloc(&b->scal, np) == cudaSuccess && dalloc(&b->partial, npart) == cudaSuccess &&
            dalloc(&b->dcount, np) == cudaSuccess && dalloc(&b->dnorm, np) == cudaSuccess &&
            dalloc(&b->st64, (size_t)b->st_total) == cudaSuccess;
  if (prec == SDME_MIXED_FP32) {
    ok = ok && dalloc(&b->st32, (size_t)b->st_total) == cudaSuccess && dalloc(&b->r32, nt) == cudaSuccess &&
         dalloc(&b->p32, nt) == cudaSuccess && dalloc(&b->q32, nt) == cudaSuccess &&
         dalloc(&b->d32, nt) == cudaSuccess && dalloc(&b->x32, nt) == cudaSuccess;
  } else {
    ok = ok && dalloc(&b->r64, nt) == cudaSuccess && dalloc(&b->p64, nt) == cudaSuccess &&
         dalloc(&b->q64, nt) == cudaSuccess && dalloc(&b->d64, nt) == cudaSuccess &&
         dalloc(&b->x64, nt) == cudaSuccess;
  }
  ok = ok && dalloc(&b->un, nt) == cudaSuccess && dalloc(&b->ahat, nt) == cudaSuccess &&
       dalloc(&b->mhat, nt) == cudaSuccess && dalloc(&b->y, nt) == cudaSuccess &&
       dalloc(&b->psi, nt) == cudaSuccess && dalloc(&b->du, nt) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&b->items_h, sizeof(PersistItem) * ((size_t)b->nelem_total + 1)) == cudaSuccess;
  ok = ok && dalloc(&b->items, (size_t)b->nelem_total) == cudaSuccess && dalloc(&b->nitems, 1) == cudaSuccess &&
       dalloc(&b->queue, 1) == cudaSuccess &&
       dalloc(&b->pprobs, np * (prec == SDME_MIXED_FP32 ? persist_prob_bytes<float>()
                                                         : persist_prob_bytes<double>())) == cudaSuccess;
  ok = ok && cudaMallocHost((void**)&b->scal_h, sizeof(PcgScalars) * np) == cudaSuccess &&
       cudaMallocHost((void**)&b->dnorm_h, sizeof(double) * np) == cudaSuccess &&
       cudaMallocHost((void**)&b->err_h, sizeof(int) * np) == cudaSuccess &&
       cudaMallocHost((void**)&b->active_h, sizeof(int) * np) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) == cudaSuccess &&
       cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) == cudaSuccess;
  if (ok) {
    // every vector starts at zero (the padding between segments stays zero)
    double* v64[] = {b->r64, b->p64, b->q64, b->d64, b->x64, b->un, b->ahat, b->mhat, b->y, b->psi, b->du};
    float* v32[] = {b->r32, b->p32, b->q32, b->d32, b->x32};
    for (double* v : v64)
      if (v) ok = ok && cudaMemsetAsync(v, 0, sizeof(double) * nt, b->stream) == cudaSuccess;
    for (float* v : v32)
      if (v) ok = ok && cudaMemsetAsync(v, 0, sizeof(float) * nt, b->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(b->info, info.data(), sizeof(BatchVecInfo) * np, cudaMemcpyHostToDevice,
                               b->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(b->cta_prob, cta_prob.data(), sizeof(int) * cta_prob.size(), cudaMemcpyHostToDevice,
                               b->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(b->err, 0, sizeof(int) * np, b->stream) == cudaSuccess &&
         cudaMemsetAsync(b->scal, 0, sizeof(PcgScalars) * np, b->stream) == cudaSuccess &&
         cudaMemsetAsync(b->dcount, 0, sizeof(unsigned int) * np, b->stream) == cudaSuccess &&
         cudaStreamSynchronize(b->stream) == cudaSuccess;
  }
  if (ok) {
    // tangent gather / scatter offset tables of the even-order problems:
    // entry (c, r, q, p) at c Nn + (r N1 + q) N0 + p from the element corner
    std::vector<int> tab;
    std::vector<int64_t> toff(np, -1);
    for (size_t i = 0; i < np; ++i) {
      const Prob& pr = b->probs[i];
      const HostMesh& h = pr.hm;
      if (pr.P % 2 != 0 || 3 * h.Nn > (int64_t)INT32_MAX) continue;
      const int n = pr.P + 1;
      toff[i] = (int64_t)tab.size();
      for (int c = 0; c < 3; ++c)
        for (int r = 0; r < n; ++r)
          for (int q = 0; q < n; ++q)
            for (int pp = 0; pp < n; ++pp)
              tab.push_back((int)(c * h.Nn + ((int64_t)r * h.N[1] + q) * h.N[0] + pp));
    }
    if (!tab.empty()) {
      ok = dalloc(&b->loc, tab.size()) == cudaSuccess &&
           cudaMemcpy(b->loc, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice) == cudaSuccess;
      for (Group& g : b->groups)
        for (HostBatchLaunch& L : g.launches)
          for (size_t k = 0; ok && k < L.pid.size(); ++k)
            if (toff[L.pid[k]] >= 0) L.mesh[k].loc = b->loc + toff[L.pid[k]];
      for (size_t i = 0; ok && i < np; ++i)
        if (toff[i] >= 0) b->probs[i].hm.loc = b->loc + toff[i];
    }
  }
  if (!ok) {
    cudaGetLastError();
    batch_free(b);
    delete b;
    return SDME_ENOMEM;
  }
  *out = b;
  return SDME_OK;
}

sdme_status sdme_batch_destroy(sdme_batch* b) {
  if (!b) return SDME_OK;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  delete b;
  return SDME_OK;
}

sdme_status sdme_batch_layout(const sdme_batch* b, int64_t* total_len, int64_t* off, int64_t* ndof) {
  if (!b) return SDME_EINVAL;
  if (total_len) *total_len = b->total;
  for (int i = 0; i < b->nprob; ++i) {
    if (off) off[i] = b->probs[i].off;
    if (ndof) ndof[i] = b->probs[i].ndof;
  }
  return SDME_OK;
}

sdme_status sdme_batch_launches(const sdme_batch* b, int64_t* launches) {
  if (!b || !launches) return SDME_EINVAL;
  *launches = b->launches;
  return SDME_OK;
}

sdme_status sdme_batch_internal_force(sdme_batch* b, const double* u_dev, double* R_dev) {
  if (!b || !u_dev || !R_dev) return SDME_EINVAL;
  B_TRY(b_residual(b, 0.0, u_dev, R_dev));
  return b_check_err(b);
}

sdme_status sdme_batch_tangent_apply(sdme_batch* b, const double* u_dev, double b1, const double* x_dev,
                                     double* y_dev) {
  if (!b || !u_dev || !x_dev || !y_dev) return SDME_EINVAL;
  B_TRY(b_residual(b, 0.0, u_dev, b->y));
  B_TRY(b_check_err(b));
  kb_mask_init<double><<<b->vec_grid, kVecThreads, 0, b->stream>>>(b->info, b->cta_prob, x_dev, y_dev);
  B_CUDA(cudaGetLastError());
  b->launches += 1;
  if (b->prec == SDME_MIXED_FP32) B_TRY((b_tangent<float, double>(b, b1, x_dev, y_dev, nullptr, nullptr)));
  else B_TRY((b_tangent<double, double>(b, b1, x_dev, y_dev, nullptr, nullptr)));
  B_CUDA(cudaStreamSynchronize(b->stream));
  return SDME_OK;
}

sdme_status sdme_batch_traction_load(sdme_batch* b, int face, const double* t_host, double* f_dev) {
  if (!b || !t_host || !f_dev || face < 0 || face > 5) return SDME_EINVAL;
  std::vector<double> f((size_t)b->total, 0.0);
  for (int i = 0; i < b->nprob; ++i) {
    const Prob& pr = b->probs[i];
    const HostElemData& h = b->groups[pr.group].tabs;
    const int P = pr.P, n = P + 1, Q = pr.Q;
    std::vector<double> I(n, 0.0);  // int_{-1}^{1} phi_j
    for (int q = 0; q < Q; ++q)
      for (int j = 0; j < n; ++j) I[j] += h.W[q] * h.B[q * n + j];
    const int axis = face / 2, side = face % 2;
    const int ta = (axis == 0) ? 1 : 0, tb = (axis == 2) ? 1 : 2;
    double hl[3];
    for (int d = 0; d < 3; ++d) hl[d] = pr.d.mesh.length[d] / pr.d.mesh.nelem[d];
    const double jac = 0.25 * hl[ta] * hl[tb];
    const int fixed = side ? pr.hm.N[axis] - 1 : 0;
    const double* t = t_host + 3 * i;
    for (int ea = 0; ea < pr.hm.ne[ta]; ++ea)
      for (int eb = 0; eb < pr.hm.ne[tb]; ++eb)
        for (int a = 0; a < n; ++a)
          for (int bq = 0; bq < n; ++bq) {
            int idx[3];
            idx[axis] = fixed;
            idx[ta] = ea * P + a;
            idx[tb] = eb * P + bq;
            const int64_t node = ((int64_t)idx[2] * pr.hm.N[1] + idx[1]) * pr.hm.N[0] + idx[0];
            const double w = jac * I[a] * I[bq];
            for (int c = 0; c < 3; ++c) f[pr.off + c * pr.hm.Nn + node] += t[c] * w;
          }
  }
  B_CUDA(cudaMemcpyAsync(f_dev, f.data(), sizeof(double) * b->total, cudaMemcpyHostToDevice, b->stream));
  B_CUDA(cudaStreamSynchronize(b->stream));
  return SDME_OK;
}

sdme_status sdme_batch_newmark_step(sdme_batch* b, sdme_state* state, double dt, const double* P_next_dev,
                                    const sdme_newton_opts* opts, sdme_step_stats* stats) {
  if (!b || !state || !state->u || !state->v || !state->a || !P_next_dev || !(dt > 0.0)) return SDME_EINVAL;
  sdme_newton_opts o{0.25, 0.5, 1e-8, 30, 1e-10, 1e-4, 20000};
  if (opts) o = *opts;
  if (!(o.beta > 0.0) || o.max_newton < 0 || o.pcg_maxit < 1) return SDME_EINVAL;
  const int np = b->nprob;
  const int64_t nt = b->total;
  const double b1 = 1.0 / (o.beta * dt * dt), b2 = 1.0 / (o.beta * dt), b3 = (1.0 - 2.0 * o.beta) / (2.0 * o.beta);
  cudaStream_t s = b->stream;
  B_CUDA(cudaMemcpyAsync(b->un, state->u, sizeof(double) * nt, cudaMemcpyDeviceToDevice, s));
  k_newmark_ahat<<<kVecGridTotal, kVecThreads, 0, s>>>(nt, b->un, state->v, state->a, b1, b2, b3, b->ahat);
  B_CUDA(cudaGetLastError());
  b->launches += 1;
  B_TRY(b_mass(b, b->ahat, b->mhat));
  kb_norm2<<<b->vec_grid, kVecThreads, 0, s>>>(b->info, b->cta_prob, P_next_dev, b->partial, b->dcount, b->dnorm);
  B_CUDA(cudaGetLastError());
  b->launches += 1;
  B_CUDA(cudaMemcpyAsync(b->dnorm_h, b->dnorm, sizeof(double) * np, cudaMemcpyDeviceToHost, s));
  B_CUDA(cudaStreamSynchronize(s));
  std::vector<double> pnorm(np), psi0(np, -1.0);
  std::vector<sdme_step_stats> st(np);
  std::vector<sdme_status> res(np, SDME_NEWTON_DIVERGED);
  for (int i = 0; i < np; ++i) {
    pnorm[i] = std::sqrt(b->dnorm_h[i]);
    std::memset(&st[i], 0, sizeof(sdme_step_stats));
    b->active_h[i] = 1;
  }
  const double inner_rtol = (b->prec == SDME_MIXED_FP32) ? o.mixed_rtol : o.pcg_rtol;
  for (int k = 0; k <= o.max_newton; ++k) {
    B_TRY(b_residual(b, b1, state->u, b->y));
    kb_residual_combine<<<b->vec_grid, kVecThreads, 0, s>>>(b->info, b->cta_prob, P_next_dev, b->mhat, b->y,
                                                            b->psi, b->partial, b->dcount, b->dnorm);
    B_CUDA(cudaGetLastError());
    b->launches += 1;
    B_CUDA(cudaMemcpyAsync(b->dnorm_h, b->dnorm, sizeof(double) * np, cudaMemcpyDeviceToHost, s));
    B_CUDA(cudaMemcpyAsync(b->err_h, b->err, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
    B_CUDA(cudaStreamSynchronize(s));
    bool jbad = false;
    for (int i = 0; i < np; ++i) jbad = jbad || b->err_h[i] != 0;
    if (jbad) B_CUDA(cudaMemsetAsync(b->err, 0, sizeof(int) * np, s));
    bool any = false;
    for (int i = 0; i < np; ++i) {
      if (!b->active_h[i]) continue;
      if (b->err_h[i]) {  // det F <= 0 somewhere in this problem: it stops here
        res[i] = SDME_NONPOSITIVE_J;
        b->active_h[i] = 0;
        continue;
      }
      const double nrm = std::sqrt(b->dnorm_h[i]);
      if (!std::isfinite(nrm)) {
        res[i] = SDME_NAN;
        b->active_h[i] = 0;
        continue;
      }
      if (psi0[i] < 0.0) {
        psi0[i] = nrm;
        st[i].residual_ref = std::max(nrm, pnorm[i]);
      }
      if (k < 33) st[i].residuals[k] = nrm;
      st[i].residual_final = nrm;
      st[i].newton_iters = k;
      if (nrm <= o.newton_tol * st[i].residual_ref) {
        res[i] = SDME_OK;
        st[i].converged = 1;
        b->active_h[i] = 0;
        continue;
      }
      if (k == o.max_newton) {
        b->active_h[i] = 0;
        continue;
      }
      any = true;
    }
    if (!any) break;
    B_CUDA(cudaMemcpyAsync(b->active, b->active_h, sizeof(int) * np, cudaMemcpyHostToDevice, s));
    B_TRY(b_pcg_dispatch(b, b1, b->psi, b->du, inner_rtol, o.pcg_maxit));
    for (int i = 0; i < np; ++i) {
      if (!b->active_h[i]) continue;
      const PcgScalars& sc = b->scal_h[i];
      if (sc.status == kPcgBreakdown) {
        res[i] = SDME_NAN;
        b->active_h[i] = 0;
      }
      if (k < 32) st[i].pcg_iters[k] = sc.iter;
      st[i].pcg_iters_total += sc.iter;
      st[i].matvecs += sc.iter;
    }
    k_axpy<double><<<kVecGridTotal, kVecThreads, 0, s>>>(nt, 1.0, b->du, state->u);
    B_CUDA(cudaGetLastError());
    b->launches += 1;
  }
  k_newmark_final<<<kVecGridTotal, kVecThreads, 0, s>>>(nt, state->u, b->ahat, b1, dt, o.gamma, state->v, state->a);
  B_CUDA(cudaGetLastError());
  b->launches += 1;
  B_CUDA(cudaStreamSynchronize(s));
  sdme_status out = SDME_OK;
  for (int i = 0; i < np; ++i) {
    st[i].residual0 = psi0[i];
    if (stats) stats[i] = st[i];
    if (out == SDME_OK && res[i] != SDME_OK) out = res[i];
  }
  return out;
}

sdme_status sdme_batch_set_persistent(sdme_batch* b, int mode, const int* kper) {
  if (!b || mode < -1 || mode > 1) return SDME_EINVAL;
  if (kper)
    for (int P = 1; P <= kMaxP; ++P) {
      const int nt = (3 * (P + 2) * (P + 2) + 31) / 32 * 32;
      if (kper[P] < 1 || kper[P] > std::min(kPersistMaxTile, 320 / nt)) return SDME_EINVAL;
    }
  if (kper) {
    for (int P = 1; P <= kMaxP; ++P) b->kper[P] = kper[P];
    std::memset(b->persist_grid_cache, 0, sizeof(b->persist_grid_cache));
  }
  b->persist_mode = mode;
  b->persist_on = mode == 1;
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  b->grun.clear();
  b->persist_grid = 0;
  return SDME_OK;
}

sdme_status sdme_batch_persistent_info(const sdme_batch* b, int* on, int kper[9], float* persist_ms,
                                       float* groups_ms, float order_ms[9]) {
  if (!b) return SDME_EINVAL;
  if (order_ms)
    for (int P = 0; P <= 8; ++P) order_ms[P] = b->persist_order_ms[P];
  if (on) *on = b->persist_on ? 1 : 0;
  if (kper)
    for (int P = 0; P <= 8; ++P) kper[P] = b->kper[P];
  if (persist_ms) *persist_ms = b->persist_ms;
  if (groups_ms) *groups_ms = b->groups_ms;
  return SDME_OK;
}

sdme_status sdme_batch_tune(sdme_batch* b, int reps, int ngroups_max, int* ngroups, int* orders, int* grids,
                            float* ms) {
  if (!b || reps < 1) return SDME_EINVAL;
  // linearisation state at u = 0 (uses the batch's scratch vectors)
  B_CUDA(cudaMemsetAsync(b->un, 0, sizeof(double) * b->total, b->stream));
  B_TRY(b_residual(b, 0.0, b->un, b->y));
  B_TRY(b_check_err(b));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  B_CUDA(cudaEventCreate(&e0));
  B_CUDA(cudaEventCreate(&e1));
  sdme_status result = SDME_OK;
  int gi = 0;
  for (Group& g : b->groups) {
    int occ = 0;
    const bool mixed = b->prec == SDME_MIXED_FP32;
    cudaError_t oe = dispatch_order(g.P, [&](auto Pc) {
      constexpr int P = decltype(Pc)::value;
      occ = mixed ? batch_tangent_occupancy<P, float, float>() : batch_tangent_occupancy<P, double, double>();
      return cudaSuccess;
    });
    (void)oe;
    std::vector<int> cand = {0};
    if (occ > 0)
      for (int mult : {1, 2, 4}) {
        const int64_t gsz = (int64_t)mult * occ * 152;
        if (gsz < g.nelem) cand.push_back((int)gsz);
      }
    float best = -1.f;
    int best_grid = 0;
    for (int grid : cand) {
      float t = 0.f;
      for (int r = -1; r < reps; ++r) {  // r = -1: warm-up launch
        if (r == 0) cudaEventRecord(e0, b->stream);
        sdme_status ts = mixed ? b_tangent_group<float, float>(b, g, 0.0, grid, b->p32, b->q32, nullptr, nullptr)
                               : b_tangent_group<double, double>(b, g, 0.0, grid, b->p64, b->q64, nullptr, nullptr);
        if (ts != SDME_OK) result = ts;
      }
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
        result = SDME_ECUDA;
        break;
      }
      t /= reps;
      if (best < 0.f || t < best) {
        best = t;
        best_grid = grid;
      }
    }
    g.grid = best_grid;
    g.tuned_ms = best;
    if (gi < ngroups_max) {
      if (orders) orders[gi] = g.P;
      if (grids) grids[gi] = g.grid;
      if (ms) ms[gi] = g.tuned_ms;
    }
    ++gi;
    if (result != SDME_OK) break;
  }
  if (ngroups) *ngroups = (int)b->groups.size();
  // the cross-order persistent operator: elements per item for each order
  // (timed on that order's problems alone), then the whole batch in one
  // launch against the sum of the per-order launches
  b->groups_ms = 0.f;
  for (const Group& g : b->groups) b->groups_ms += g.tuned_ms;
  if (result == SDME_OK && b->persist_mode != 0) {
    const bool mixed = b->prec == SDME_MIXED_FP32;
    auto time_persist = [&](float* out) -> sdme_status {
      // every problem running, counters at zero (the next PCG initialises them again)
      B_CUDA(cudaMemsetAsync(b->scal, 0, sizeof(PcgScalars) * b->nprob, b->stream));
      float t = 0.f;
      for (int r = -1; r < reps; ++r) {
        if (r == 0) B_CUDA(cudaEventRecord(e0, b->stream));
        B_TRY((mixed ? b_persist_launch<float, float>(b, b->p32, b->q32, b->partial, b->scal, true)
                     : b_persist_launch<double, double>(b, b->p64, b->q64, b->partial, b->scal, true)));
      }
      B_CUDA(cudaEventRecord(e1, b->stream));
      B_CUDA(cudaEventSynchronize(e1));
      B_CUDA(cudaEventElapsedTime(&t, e0, e1));
      *out = t / reps;
      return SDME_OK;
    };
    for (Group& g : b->groups) {
      const int nt = (3 * (g.P + 2) * (g.P + 2) + 31) / 32 * 32;
      const int kmax = std::max(1, std::min(kPersistMaxTile, 320 / nt));
      float best = -1.f;
      int bestk = 1;
      for (int k = 1; k <= kmax && result == SDME_OK; ++k) {
        b->kper[g.P] = k;
        std::memset(b->persist_grid_cache, 0, sizeof(b->persist_grid_cache));
        float t = 0.f;
        result = b_persist_items(b, nullptr, 0.0, g.P);
        if (result == SDME_OK) result = b_persist_grid(b);
        if (result == SDME_OK) result = time_persist(&t);
        if (result == SDME_OK && (best < 0.f || t < best)) {
          best = t;
          bestk = k;
        }
      }
      b->kper[g.P] = bestk;
      b->persist_order_ms[g.P] = best;
    }
    std::memset(b->persist_grid_cache, 0, sizeof(b->persist_grid_cache));
    if (result == SDME_OK) result = b_persist_items(b, nullptr, 0.0);
    if (result == SDME_OK) result = b_persist_grid(b);
    if (result == SDME_OK) result = time_persist(&b->persist_ms);
    b->persist_on = result == SDME_OK && (b->persist_mode == 1 || b->persist_ms < b->groups_ms);
    b->persist_b1 = -1.0;   // rebuilt with the solve's b1
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the tuning launches wrote into q: clear it for the next PCG
  if (b->q32) cudaMemsetAsync(b->q32, 0, sizeof(float) * b->total, b->stream);
  if (b->q64) cudaMemsetAsync(b->q64, 0, sizeof(double) * b->total, b->stream);
  B_CUDA(cudaStreamSynchronize(b->stream));
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  return result;
}

}  // extern "C"
