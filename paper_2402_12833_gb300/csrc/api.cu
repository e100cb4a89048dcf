// C ABI of libmpcg: hierarchy setup (Section 2.1) and the additive-MG MPCG
// solver (Section 2.2, Algorithm 1), FP64 and FP32-bulk mixed precision.
//
// One solver iteration is captured once as a CUDA graph whose body sits in a
// device-side while loop (a conditional graph node): the convergence kernel
// clears the loop condition, so a whole solve is a single graph launch with
// no host round trip per iteration.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "amg.h"
#include "kernels.cuh"
#include "tune.h"

using namespace mpcg;

namespace {

thread_local std::string g_err;

void set_err(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      set_err("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? MPCG_ERR_OOM : MPCG_ERR_CUDA;               \
    }                                                                                      \
  } while (0)

#define CKS(expr)                              \
  do {                                         \
    mpcg_status s_ = (expr);                   \
    if (s_ != MPCG_OK) return s_;              \
  } while (0)

// A sparse matrix of an algebraic hierarchy in device memory (EllDev layout);
// the FP32 values exist once the mixed-precision solver is built.
struct EllLevel {
  int rows = 0, cols = 0, nslices = 0, lg = 0;
  int* sptr = nullptr;
  int* col = nullptr;
  double* v64 = nullptr;
  float* v32 = nullptr;
  dw* vdw = nullptr;   // double-word values (MPCG_FP64_DW)
  long long nent = 0;   // stored entries, padding included
};

template <typename T>
EllDev<T> ell_of(const EllLevel& E);
template <>
EllDev<double> ell_of<double>(const EllLevel& E) { return {E.rows, E.cols, E.nslices, E.lg, E.sptr, E.col, E.v64}; }
template <>
EllDev<float> ell_of<float>(const EllLevel& E) { return {E.rows, E.cols, E.nslices, E.lg, E.sptr, E.col, E.v32}; }
template <>
EllDev<dw> ell_of<dw>(const EllLevel& E) { return {E.rows, E.cols, E.nslices, E.lg, E.sptr, E.col, E.vdw}; }

struct Level {
  GridDesc g;
  int nplanes = 0;   // stencil planes: ncomp * 3^dim
  int ndinv = 0;     // inverse-diagonal planes: ncomp
  double* st64 = nullptr;
  float* st32 = nullptr;
  float* sth32 = nullptr;        // scalar grids: the symmetric half of st32 (FP32 SpMM and smoothing)
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  dw* stdw = nullptr;            // double-word copies (MPCG_FP64_DW)
  dw* dinvdw = nullptr;
  float* kq32 = nullptr;         // fine grid: element coefficients in use (matrix-free FP32 operator), or null
  float* kq32_store = nullptr;   // their storage (kept across detach / attach)
  // algebraic hierarchies: the grid's operator, P_j (grid j-1 -> j) and R_j = P_j^T
  EllLevel eA, eP, eR;
};

struct Alloc {
  std::vector<void*> ptrs;
  template <typename P>
  mpcg_status get(P** p, size_t count, cudaStream_t s) {
    void* q = nullptr;
    const size_t bytes = count * sizeof(P);
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      set_err("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
      return MPCG_ERR_OOM;
    }
    ptrs.push_back(q);
    e = cudaMemsetAsync(q, 0, bytes ? bytes : 16, s);
    if (e != cudaSuccess) {
      set_err("cudaMemsetAsync failed: %s", cudaGetErrorString(e));
      return MPCG_ERR_CUDA;
    }
    *p = (P*)q;
    return MPCG_OK;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

template <typename T>
struct Solver {
  bool built = false;
  int C = 0, m = 0, hist_cap = 0;
  Alloc mem, hist_mem;
  T* rlev[kMaxLevels] = {};
  T* zc[kMaxLevels] = {};
  T* tmp[kMaxLevels] = {};
  T* tmp2[kMaxLevels] = {};
  T *x = nullptr, *r = nullptr, *b = nullptr, *Z = nullptr, *AZ = nullptr;
  T* Zmg = nullptr;   // the per-grid columns when they are summed into one
  Window<T> win = {};
  DevState* state = nullptr;
  double *part_res = nullptr, *part_zaz = nullptr, *part_W = nullptr, *part_G = nullptr, *part_r = nullptr;
  double* small_scratch = nullptr;   // reduced values of the small solves
  unsigned* counters = nullptr;      // last-block counters of small_beta / small_alpha
  int* flag = nullptr;               // "some problem still running" (batched loop condition)
  int* kdone = nullptr;              // gathered (iterations, done) per problem
  double *res_hist = nullptr, *alpha_hist = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = false;
  // x starts at zero and r = b, |r|^2, |b|^2 partials are written before the
  // prologue (the inner solves of the mixed-precision refinement)
  bool zero_start = false;
  long long prologue_launches = 0, body_launches = 0;
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    use_graph = false;
  }
  void release() {
    drop_graph();
    mem.release();
    hist_mem.release();
    built = false;
    hist_cap = 0;
  }
};

enum KClass {
  K_PACK, K_RESIDUAL, K_INIT, K_RESTRICT, K_COARSE, K_PROLONG, K_JACOBI, K_SPMM, K_GRAM, K_BETA, K_ORTH,
  K_ALPHA, K_UPDATE, K_CHECK, K_AUX, K_NET, K_OGRAM, K_COUNT
};
const char* const kClassNames[K_COUNT] = {"pack", "residual", "init", "restrict", "coarse_solve", "prolong",
                                          "jacobi", "spmm", "gram_window", "small_beta", "orth_update",
                                          "small_alpha", "update_xr", "check", "aux", "net", "orth_gram"};

// Launch accounting and optional per-launch CUDA-event timing (direct
// launches only; never active while a graph is captured).
struct Profiler {
  bool on = false;
  long long* target = nullptr;      // launch counter currently charged
  long long live = 0;               // launches executed by the current call
  long long count[K_COUNT] = {};
  double ms[K_COUNT] = {};
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, size_t>> pending;
  std::vector<std::pair<int, float>> trace;   // (class, ms) of every timed launch, in order
  size_t used = 0;
  void begin(int cls, cudaStream_t s) {
    ++*(target ? target : &live);
    if (!on) return;
    if (used + 2 > pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        pool.push_back(e);
      }
    }
    cudaEventRecord(pool[used], s);
    pending.push_back({cls, used});
    used += 2;
  }
  void end(cudaStream_t s) {
    if (on) cudaEventRecord(pool[pending.back().second + 1], s);
  }
  void flush() {
    for (auto& pr : pending) {
      float t = 0.f;
      cudaEventSynchronize(pool[pr.second + 1]);
      cudaEventElapsedTime(&t, pool[pr.second], pool[pr.second + 1]);
      ms[pr.first] += t;
      count[pr.first] += 1;
      trace.push_back({pr.first, t});
    }
    pending.clear();
    used = 0;
  }
  void reset() {
    trace.clear();
    pending.clear();
    used = 0;
    live = 0;
    for (int i = 0; i < K_COUNT; ++i) count[i] = 0, ms[i] = 0.0;
  }
  void release() {
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

}  // namespace

#define LAUNCH(h, cls, s, ...)        \
  do {                                \
    (h)->prof.begin((cls), (s));      \
    __VA_ARGS__;                      \
    (h)->prof.end((s));               \
  } while (0)

// identity of a hierarchy for caches that outlive a call (never reused)
static long long next_hierarchy_uid() {
  static std::atomic<long long> n{0};
  return ++n;
}

struct mg_hierarchy {
  long long uid = next_hierarchy_uid();
  long long graph_gen = 0;     // bumped whenever the mixed-precision graph is dropped
  int device = 0;
  int dim = 2, levels = 1;
  int nodes = 0;               // fine-grid nodes per side, boundary included
  int nb = 1;                  // problems in the batch (same grid, own operators)
  int* active = nullptr;       // mixed path: problems still refining
  mpcg_options opt;
  cudaStream_t stream = 0;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side[kMaxLevels] = {};   // branches of the MG chain: fine smoothing, one per coarse grid
  cudaEvent_t ev_fork = nullptr, ev_fine = nullptr;
  cudaEvent_t ev_r[kMaxLevels] = {}, ev_sm[kMaxLevels] = {};
  double* A0inv = nullptr;
  Level lev[kMaxLevels];
  double* L0 = nullptr;
  double* rdiag0 = nullptr;
  int n0 = 0;
  int* info = nullptr;
  bool have32 = false;
  Alloc mem;
  Solver<double> s64;
  Solver<float> s32;
  Solver<dw> sdw;            // FP64 data, double-word arithmetic (MPCG_FP64_DW)
  bool havedw = false;
  double *b64 = nullptr, *x64 = nullptr, *r64 = nullptr, *nrm = nullptr, *part_mix = nullptr;
  int* xnz = nullptr;        // per problem: the packed FP64 iterate may be nonzero
  double* stage = nullptr;   // 2 n doubles: staging for host b and x
  // mixed precision as one graph (refinement loop on the device)
  int* mix = nullptr;        // per problem: inner iterations, status, active
  int* outer = nullptr;      // refinement steps taken
  cudaGraph_t mgraph = nullptr;
  cudaGraphExec_t mexec = nullptr;
  double mg_rtol = -1.0;
  int mg_maxit = -1, mg_hist = -1;
  long long mg_head = 0, mg_tail = 0, mg_iprol = 0, mg_ibody = 0;   // launches per part
  Profiler prof;
  bool force_direct = false;
  long long last_launches = 0;
  // learned search column (extension): appended as column `levels`
  bool net_on = false;
  float* net_wq = nullptr;     // bfloat16-valued weights
  float* net_c = nullptr;      // coefficient channel on the fine grid
  NetActs net_acts = {};       // inference activations
  int* net_err = nullptr;      // set by the tensor-core inference kernel on a timed-out wait
  unsigned char* net_wtc = nullptr;   // weights packed for the tensor-core kernel
  Alloc net_mem;
  // algebraic hierarchy (flat grids, ELL operators); host copies of its
  // matrices by grid index: A[j], P[j] (j >= 1), aggregates of grid j (j >= 1)
  bool algebraic = false;
  std::vector<mpcg::amg::Csr> amgA, amgP;
  std::vector<std::vector<int>> amgAgg;
};

namespace {

// Graphs that hold the mixed-precision solves of several hierarchies (the
// size classes of a batch of uneven problems, mpcg_solve_batched_graph),
// keyed by the classes' identities, graph generations and history
// capacities, the tolerance and the iteration limit.
struct ClassGraph {
  std::vector<long long> uid, gen;
  std::vector<int> hist;
  double rtol = 0.0;
  int maxit = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};
std::mutex g_class_graph_mu;
std::vector<ClassGraph> g_class_graphs;
constexpr size_t kMaxClassGraphs = 8;

void destroy_class_graph(ClassGraph& e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.graph) cudaGraphDestroy(e.graph);
  e.exec = nullptr;
  e.graph = nullptr;
}

// Drop every cached class graph that contains hierarchy `uid`.
void purge_class_graphs(long long uid) {
  std::lock_guard<std::mutex> lk(g_class_graph_mu);
  for (size_t i = 0; i < g_class_graphs.size();) {
    auto& u = g_class_graphs[i].uid;
    if (std::find(u.begin(), u.end(), uid) != u.end()) {
      destroy_class_graph(g_class_graphs[i]);
      g_class_graphs.erase(g_class_graphs.begin() + i);
    } else {
      ++i;
    }
  }
}

template <typename T>
const T* st_of(const Level& L);
template <>
const double* st_of<double>(const Level& L) { return L.st64; }
template <>
const float* st_of<float>(const Level& L) { return L.st32; }
template <>
const dw* st_of<dw>(const Level& L) { return L.stdw; }
template <typename T>
const T* dinv_of(const Level& L);
template <>
const double* dinv_of<double>(const Level& L) { return L.dinv64; }
template <>
const float* dinv_of<float>(const Level& L) { return L.dinv32; }
template <>
const dw* dinv_of<dw>(const Level& L) { return L.dinvdw; }

template <typename T>
mpcg_status build_solver(mg_hierarchy* h, Solver<T>& S) {
  if (S.built) return MPCG_OK;
  cudaStream_t s = h->stream;
  const int J = h->levels - 1;
  const GridDesc& gf = h->lev[J].g;
  S.C = (h->opt.sum_columns || h->opt.vcycle) ? 1 : h->levels + (h->net_on ? 1 : 0);
  S.m = h->opt.m;
  // the FP32 solver only runs the inner solves of the refinement, which
  // start from zero with r = b written by launch_start_inner
  S.zero_start = std::is_same<T, float>::value;
  const int C = S.C;
  const size_t nb = (size_t)h->nb;   // all buffers hold the whole batch
  CKS(S.mem.get(&S.x, gf.cp, s));
  CKS(S.mem.get(&S.r, gf.cp, s));
  CKS(S.mem.get(&S.b, gf.cp, s));
  CKS(S.mem.get(&S.Z, (size_t)C * gf.cp, s));
  if (h->opt.sum_columns) CKS(S.mem.get(&S.Zmg, (size_t)h->levels * gf.cp, s));
  CKS(S.mem.get(&S.AZ, (size_t)C * gf.cp, s));
  for (int j = 0; j < S.m; ++j) {
    CKS(S.mem.get(&S.win.P[j], (size_t)C * gf.cp, s));
    CKS(S.mem.get(&S.win.AP[j], (size_t)C * gf.cp, s));
  }
  for (int j = 0; j <= J; ++j) {
    const GridDesc& g = h->lev[j].g;
    if (j < J) {
      CKS(S.mem.get(&S.rlev[j], g.cp, s));
      CKS(S.mem.get(&S.zc[j], (size_t)(j + 1) * g.cp, s));
    }
    if (h->opt.nu > 2 || (g.ncomp > 1 && h->opt.nu > 1) || h->opt.vcycle) {   // V-cycle: defects
      CKS(S.mem.get(&S.tmp[j], g.cp, s));
      CKS(S.mem.get(&S.tmp2[j], g.cp, s));
    }
  }
  CKS(S.mem.get(&S.state, nb, s));
  // partial-sum slots for the most blocks a tuned launch shape may take
  // (the autotuner can change the shapes after the buffers exist)
  const size_t sbc = (size_t)stream_blocks_cap(gf), gcc = (size_t)gram_chunks_cap(gf);
  CKS(S.mem.get(&S.part_res, nb * 2 * sbc, s));
  CKS(S.mem.get(&S.part_zaz, nb * C * sbc, s));
  CKS(S.mem.get(&S.part_W, nb * S.m * C * C * gcc, s));
  CKS(S.mem.get(&S.part_G, nb * (C * (C + 1) / 2 + C) * sbc, s));
  CKS(S.mem.get(&S.part_r, nb * sbc, s));
  CKS(S.mem.get(&S.small_scratch, nb * kSmallScratch, s));
  CKS(S.mem.get(&S.counters, 2 * nb, s));
  CKS(S.mem.get(&S.flag, 1, s));
  CKS(S.mem.get(&S.kdone, 2 * nb, s));
  S.built = true;
  return MPCG_OK;
}

template <typename T>
mpcg_status ensure_hist(mg_hierarchy* h, Solver<T>& S, int maxit) {
  if (S.hist_cap >= maxit + 1) return MPCG_OK;
  S.drop_graph();
  S.hist_mem.release();
  int cap = 64;
  while (cap < maxit + 1) cap *= 2;
  CKS(S.hist_mem.get(&S.res_hist, (size_t)cap * h->nb, h->stream));
  CKS(S.hist_mem.get(&S.alpha_hist, (size_t)cap * S.C * h->nb, h->stream));
  S.hist_cap = cap;
  return MPCG_OK;
}

// nu damped-Jacobi sweeps from zero on grid j: rr -> out.
// k multicoloured SSOR steps on grid j for the right-hand side rr, in place
// on x (a forward sweep over the 2^dim colours, then a backward one).
// With omega = 1 a colour updated twice in a row (the turn of each step,
// K-1 then K-1, and colour 0 between steps) gets an exactly zero second
// update: unknowns of one colour do not couple, so the first update already
// zeroed the colour's residual; those launches are skipped (the result moves
// by rounding only).
template <typename T>
void enqueue_ssor_steps(mg_hierarchy* h, int j, const T* rr, T* x, int k, const DevState* state, cudaStream_t s) {
  const Level& L = h->lev[j];
  const int K = 1 << L.g.dim;
  const bool skip_repeat = h->opt.ssor_omega == 1.0;
  int last = -1;
  auto update = [&](int c) {
    if (skip_repeat && c == last) return;
    LAUNCH(h, K_JACOBI, s, launch_gs_colour<T>(L.g, st_of<T>(L), rr, x, c, h->opt.ssor_omega, state, s));
    last = c;
  };
  for (int step = 0; step < k; ++step) {
    for (int c = 0; c < K; ++c) update(c);
    for (int c = K - 1; c >= 0; --c) update(c);
  }
}

// Damped-Jacobi launch of a scalar stencil grid (modes as launch_jacobi):
// FP32 reads the symmetric half where the grid has one.
template <typename T>
void jacobi_of(const Level& L, const T* st, const T* di, const T* rr, const T* sin, T* out, int mode,
               const DevState* state, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (L.sth32) {
      launch_jacobi_sym(L.g, L.sth32, di, rr, sin, out, mode, state, s);
      return;
    }
  }
  launch_jacobi<T>(L.g, st, di, rr, sin, out, mode, state, s);
}

template <typename T>
void enqueue_smooth(mg_hierarchy* h, Solver<T>& S, int j, const T* rr, T* out, const DevState* state,
                    cudaStream_t s) {
  const Level& L = h->lev[j];
  const T* st = st_of<T>(L);
  const T* di = dinv_of<T>(L);
  const int nu = h->opt.nu;
  if (h->algebraic) {   // damped Jacobi with the grid's sparse operator
    const EllDev<T> E = ell_of<T>(L.eA);
    const long long G = L.g.G;
    if (nu <= 2) {
      LAUNCH(h, K_JACOBI, s, launch_ell_jacobi<T>(E, di + G, rr + G, nullptr, out + G, nu - 1, state, s));
      return;
    }
    T* a = S.tmp[j];
    T* b = S.tmp2[j];
    LAUNCH(h, K_JACOBI, s, launch_ell_jacobi<T>(E, di + G, rr + G, nullptr, a + G, 1, state, s));
    for (int k = 3; k <= nu; ++k) {
      T* o = k == nu ? out : b;
      LAUNCH(h, K_JACOBI, s, launch_ell_jacobi<T>(E, di + G, rr + G, a + G, o + G, 2, state, s));
      T* t = a;
      a = b;
      b = t;
    }
    return;
  }
  if (h->opt.smoother == MPCG_SMOOTHER_SSOR) {   // nu SSOR steps from zero
    cudaMemsetAsync(out, 0, sizeof(T) * L.g.cp, s);
    enqueue_ssor_steps<T>(h, j, rr, out, nu, state, s);
    return;
  }
  if (L.g.ncomp > 1) {
    // block Jacobi: s = D^-1 r, then nu - 1 sweeps t = r - A s, s += D^-1 t
    // (the update is pointwise, so it runs in place)
    T* sv = nu == 1 ? out : S.tmp[j];
    T* t = S.tmp2[j];
    LAUNCH(h, K_JACOBI, s, launch_vblock<T>(L.g, di, rr, nullptr, sv, state, s));
    // the last sweep writes `out`, not s: one fused pass on grids of at
    // least 2^17 nodes (the fine grid of the 65^3 problem); on smaller grids
    // its three components per thread leave too few threads (measured
    // 28-30 us against 17-19 us for the two launches)
    const bool fuse = L.g.cstride >= (1LL << 17);
    for (int k = 2; k <= nu; ++k) {
      if (k == nu && fuse) {
        LAUNCH(h, K_JACOBI, s, launch_vres_block<T>(L.g, st, rr, sv, di, out, state, s));
      } else {
        LAUNCH(h, K_JACOBI, s, launch_vres<T>(L.g, st, rr, sv, t, state, s));
        LAUNCH(h, K_JACOBI, s, launch_vblock<T>(L.g, di, t, sv, k == nu ? out : sv, state, s));
      }
    }
    return;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (nu == 2 && L.kq32) {   // fine grid with the matrix-free operator
      LAUNCH(h, K_JACOBI, s, launch_jacobi_mf(L.g, L.kq32, di, rr, out, state, s));
      return;
    }
  }
  if (nu == 1) {
    LAUNCH(h, K_JACOBI, s, jacobi_of<T>(L, st, di, rr, nullptr, out, 0, state, s));
  } else if (nu == 2) {
    LAUNCH(h, K_JACOBI, s, jacobi_of<T>(L, st, di, rr, nullptr, out, 1, state, s));
  } else {
    T* a = S.tmp[j];
    T* b = S.tmp2[j];
    LAUNCH(h, K_JACOBI, s, jacobi_of<T>(L, st, di, rr, nullptr, a, 1, state, s));
    for (int k = 3; k <= nu; ++k) {
      T* o = k == nu ? out : b;
      LAUNCH(h, K_JACOBI, s, jacobi_of<T>(L, st, di, rr, a, o, 2, state, s));
      T* t = a;
      a = b;
      b = t;
    }
  }
}

// The additive structure makes the level corrections independent once the
// residual has been restricted (Section 2.1): the fine-grid smoothing (which
// needs only r) runs on one side stream, and every coarse grid's smoothing on
// a side stream of its own, starting as soon as its restricted residual
// exists, while the main stream carries the restriction chain, the coarse
// solve and the prolongation chain.  Under graph capture the side streams
// become parallel graph branches.
template <typename T>
void enqueue_mg_algebraic(mg_hierarchy* h, Solver<T>& S, const T* r, T* Z, const DevState* state, cudaStream_t s);

template <typename T>
void enqueue_mg(mg_hierarchy* h, Solver<T>& S, const T* r, T* Z, const DevState* state, cudaStream_t s) {
  if (h->algebraic) {
    enqueue_mg_algebraic<T>(h, S, r, Z, state, s);
    return;
  }
  const int J = h->levels - 1;
  if (J == 0) {
    LAUNCH(h, K_COARSE, s, launch_coarse_solve<T>(h->lev[0].g, h->A0inv, r, Z, state, s));
    return;
  }
  // a profiled solve keeps every launch on one stream so that each event
  // pair brackets exactly one kernel running alone
  cudaStream_t s2 = h->prof.on ? s : h->side[0];
  cudaEventRecord(h->ev_fork, s);
  cudaStreamWaitEvent(s2, h->ev_fork, 0);
  enqueue_smooth<T>(h, S, J, r, Z + (size_t)J * h->lev[J].g.cp, state, s2);
  cudaEventRecord(h->ev_fine, s2);
  // grids of at most kTailPoints padded points (scalar unknowns, two sweeps)
  // go through one single-block launch: their restrictions, smoothings and
  // the coarse solve are latency-bound as separate launches
  int jt = -1;
  if (h->lev[0].g.ncomp == 1 && h->opt.nu == 2 && h->opt.smoother == MPCG_SMOOTHER_JACOBI)
    for (int j = 0; j < J; ++j)
      if (h->lev[j].g.npts <= kTailPoints) jt = j;
  const T* rj = r;
  for (int j = J; j >= (jt >= 0 ? jt + 2 : 1); --j) {
    LAUNCH(h, K_RESTRICT, s, launch_restrict<T>(h->lev[j].g, h->lev[j - 1].g, rj, S.rlev[j - 1], state, s));
    rj = S.rlev[j - 1];
    if (j - 1 >= 1) {   // smoothing of grid j-1 can start now, on its own branch
      cudaStream_t s3 = h->prof.on ? s : h->side[j - 1];
      cudaEventRecord(h->ev_r[j - 1], s);
      cudaStreamWaitEvent(s3, h->ev_r[j - 1], 0);
      enqueue_smooth<T>(h, S, j - 1, S.rlev[j - 1], S.zc[j - 1] + (size_t)(j - 1) * h->lev[j - 1].g.cp, state, s3);
      cudaEventRecord(h->ev_sm[j - 1], s3);
    }
  }
  if (jt >= 0) {
    GridDesc tg[kMaxLevels];
    const T* tst[kMaxLevels];
    const T* tdi[kMaxLevels];
    T* tr[kMaxLevels];
    T* tz[kMaxLevels];
    for (int j = 0; j <= jt + 1; ++j) {
      tg[j] = h->lev[j].g;
      tst[j] = st_of<T>(h->lev[j]);
      tdi[j] = dinv_of<T>(h->lev[j]);
      tr[j] = j <= jt ? S.rlev[j] : nullptr;
      tz[j] = j <= jt ? S.zc[j] + (size_t)j * h->lev[j].g.cp : nullptr;
    }
    LAUNCH(h, K_COARSE, s, launch_coarse_tail<T>(jt, tg, tst, tdi, tr, tz, rj, h->A0inv, state, s));
  } else {
    LAUNCH(h, K_COARSE, s, launch_coarse_solve<T>(h->lev[0].g, h->A0inv, S.rlev[0], S.zc[0], state, s));
  }
  // every grid's correction straight to the fine grid in one launch
  const T* src[kMaxLevels];
  GridDesc gcs[kMaxLevels];
  for (int j = 0; j < J; ++j) {
    if (j >= 1 && j > jt) cudaStreamWaitEvent(s, h->ev_sm[j], 0);
    src[j] = S.zc[j] + (size_t)j * h->lev[j].g.cp;
    gcs[j] = h->lev[j].g;
  }
  LAUNCH(h, K_PROLONG, s, launch_prolong_all<T>(h->lev[J].g, src, gcs, J, Z, state, s));
  cudaStreamWaitEvent(s, h->ev_fine, 0);
}

// The additive corrections on an algebraic hierarchy, with the branch
// structure of the structured one: the fine smoothing and each coarse grid's
// smoothing on side streams, the restriction chain R_j = P_j^T and the coarse
// solve on the main stream.  The prolongation is a cascade: P_k lifts all k
// columns that have reached grid k-1 (the corrections of grids 0 .. k-1) in
// one block SpMM, so every P_k is read once per iteration; grid j's buffer
// zc[j] holds columns 0 .. j, column j being its own smoothed correction.
template <typename T>
void enqueue_mg_algebraic(mg_hierarchy* h, Solver<T>& S, const T* r, T* Z, const DevState* state, cudaStream_t s) {
  const int J = h->levels - 1;
  if (J == 0) {
    LAUNCH(h, K_COARSE, s, launch_coarse_solve<T>(h->lev[0].g, h->A0inv, r, Z, state, s));
    return;
  }
  cudaStream_t s2 = h->prof.on ? s : h->side[0];
  cudaEventRecord(h->ev_fork, s);
  cudaStreamWaitEvent(s2, h->ev_fork, 0);
  enqueue_smooth<T>(h, S, J, r, Z + (size_t)J * h->lev[J].g.cp, state, s2);
  cudaEventRecord(h->ev_fine, s2);
  const T* rj = r;
  for (int j = J; j >= 1; --j) {
    const GridDesc& gf = h->lev[j].g;
    const GridDesc& gc = h->lev[j - 1].g;
    LAUNCH(h, K_RESTRICT, s,
           launch_ell_spmm<T>(ell_of<T>(h->lev[j].eR), rj + gf.G, gf.cp, S.rlev[j - 1] + gc.G, gc.cp, 1, nullptr, 0,
                              state, s));
    rj = S.rlev[j - 1];
    if (j - 1 >= 1) {
      cudaStream_t s3 = h->prof.on ? s : h->side[j - 1];
      cudaEventRecord(h->ev_r[j - 1], s);
      cudaStreamWaitEvent(s3, h->ev_r[j - 1], 0);
      enqueue_smooth<T>(h, S, j - 1, S.rlev[j - 1], S.zc[j - 1] + (size_t)(j - 1) * gc.cp, state, s3);
      cudaEventRecord(h->ev_sm[j - 1], s3);
    }
  }
  LAUNCH(h, K_COARSE, s, launch_coarse_solve<T>(h->lev[0].g, h->A0inv, S.rlev[0], S.zc[0], state, s));
  for (int k = 1; k <= J; ++k) {
    if (k - 1 >= 1) cudaStreamWaitEvent(s, h->ev_sm[k - 1], 0);
    const GridDesc& gc = h->lev[k - 1].g;
    const GridDesc& gk = h->lev[k].g;
    T* dst = k < J ? S.zc[k] : Z;
    LAUNCH(h, K_PROLONG, s,
           launch_ell_spmm<T>(ell_of<T>(h->lev[k].eP), S.zc[k - 1] + gc.G, gc.cp, dst + gk.G, gk.cp, k, nullptr, 0,
                              state, s));
  }
  cudaStreamWaitEvent(s, h->ev_fine, 0);
}

// r = b - A x on the fine grid (stored stencil or sparse operator).
template <typename T>
void launch_fine_residual(mg_hierarchy* h, const T* b, const T* x, T* r, double* part, cudaStream_t s,
                          const int* xnz) {
  const Level& L = h->lev[h->levels - 1];
  if (h->algebraic)
    launch_ell_residual<T>(ell_of<T>(L.eA), b + L.g.G, x + L.g.G, r + L.g.G, part, stream_blocks(L.g), s, xnz);
  else
    launch_residual<T>(L.g, st_of<T>(L), b, x, r, part, s, xnz);
}

// One damped-Jacobi sweep on grid j (stored stencil or sparse operator),
// modes as launch_jacobi: 0 xout = dinv g, 1 two sweeps from zero,
// 2 xout = xin + dinv (g - A xin).
template <typename T>
void jacobi_sweep(mg_hierarchy* h, int j, const T* g, const T* xin, T* xout, int mode, const DevState* state,
                  cudaStream_t s) {
  const Level& L = h->lev[j];
  if (h->algebraic) {
    const long long G = L.g.G;
    LAUNCH(h, K_JACOBI, s,
           launch_ell_jacobi<T>(ell_of<T>(L.eA), dinv_of<T>(L) + G, g + G, xin ? xin + G : nullptr, xout + G, mode,
                                state, s));
  } else {
    LAUNCH(h, K_JACOBI, s, jacobi_of<T>(L, st_of<T>(L), dinv_of<T>(L), g, xin, xout, mode, state, s));
  }
}

// k smoothing steps of the V-cycle on grid j for the right-hand side g, in
// place on x, from zero when `zero` (x need not be cleared then): SSOR
// steps, or damped-Jacobi sweeps alternating between x and tmp2[j] (the
// last one lands in x).
template <typename T>
void enqueue_vsmooth(mg_hierarchy* h, Solver<T>& S, int j, const T* g, T* x, int k, bool zero, const DevState* state,
                     cudaStream_t s) {
  const Level& L = h->lev[j];
  if (h->opt.smoother == MPCG_SMOOTHER_SSOR) {
    if (zero) cudaMemsetAsync(x, 0, sizeof(T) * L.g.cp, s);
    enqueue_ssor_steps<T>(h, j, g, x, k, state, s);
    return;
  }
  int left = k;
  if (zero) {
    jacobi_sweep<T>(h, j, g, nullptr, x, k >= 2 ? 1 : 0, state, s);
    left -= k >= 2 ? 2 : 1;
  }
  T* cur = x;
  for (; left > 0; --left) {
    T* dst = cur == x ? S.tmp2[j] : x;
    jacobi_sweep<T>(h, j, g, cur, dst, 2, state, s);
    cur = dst;
  }
  if (cur != x) cudaMemcpyAsync(x, cur, sizeof(T) * L.g.cp, cudaMemcpyDeviceToDevice, s);
}

// The multiplicative V(nu, nu) cycle from zero for the right-hand side r,
// into out (Section 3's MG(V) preconditioner): on every grid from the
// finest down, nu smoothing steps (SSOR, or damped Jacobi), the defect and
// its restriction; the exact coarse solve; on the way up the prolongated
// correction and nu smoothing steps.  Grid j < J keeps its right-hand side
// in rlev[j], its iterate in zc[j] and its defect in tmp[j].
template <typename T>
void enqueue_vcycle(mg_hierarchy* h, Solver<T>& S, const T* r, T* out, const DevState* state, cudaStream_t s) {
  const int J = h->levels - 1;
  const int nu = h->opt.nu;
  auto rhs = [&](int j) -> const T* { return j == J ? r : S.rlev[j]; };
  auto it = [&](int j) -> T* { return j == J ? out : S.zc[j]; };
  for (int j = J; j >= 1; --j) {
    const Level& L = h->lev[j];
    const GridDesc& gc = h->lev[j - 1].g;
    enqueue_vsmooth<T>(h, S, j, rhs(j), it(j), nu, true, state, s);
    if (h->algebraic) {
      const long long G = L.g.G;
      LAUNCH(h, K_RESIDUAL, s,
             launch_ell_defect<T>(ell_of<T>(L.eA), rhs(j) + G, it(j) + G, S.tmp[j] + G, state, s));
      LAUNCH(h, K_RESTRICT, s,
             launch_ell_spmm<T>(ell_of<T>(L.eR), S.tmp[j] + G, L.g.cp, S.rlev[j - 1] + gc.G, gc.cp, 1, nullptr, 0,
                                state, s));
    } else {
      LAUNCH(h, K_RESIDUAL, s, launch_defect<T>(L.g, st_of<T>(L), rhs(j), it(j), S.tmp[j], state, s));
      LAUNCH(h, K_RESTRICT, s, launch_restrict<T>(L.g, gc, S.tmp[j], S.rlev[j - 1], state, s));
    }
  }
  LAUNCH(h, K_COARSE, s, launch_coarse_solve<T>(h->lev[0].g, h->A0inv, S.rlev[0], it(0), state, s));
  for (int j = 1; j <= J; ++j) {
    const Level& L = h->lev[j];
    const GridDesc& gc = h->lev[j - 1].g;
    if (h->algebraic)
      LAUNCH(h, K_PROLONG, s,
             launch_ell_spmv_add<T>(ell_of<T>(L.eP), it(j - 1) + gc.G, it(j) + L.g.G, state, s));
    else
      LAUNCH(h, K_PROLONG, s, launch_prolong_add<T>(gc, L.g, it(j - 1), it(j), state, s));
    enqueue_vsmooth<T>(h, S, j, rhs(j), it(j), nu, false, state, s);
  }
}

template <typename T>
void enqueue_any(mg_hierarchy* h, Solver<T>& S, cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s);

template <typename T>
void enqueue_prologue(mg_hierarchy* h, Solver<T>& S, cudaGraphConditionalHandle cond, int use_cond,
                      cudaStream_t s) {
  const Level& L = h->lev[h->levels - 1];
  // a solve from a zero iterate has r = b, written by its start kernel
  // the FP64 iterate was packed with its nonzero flag (a zero x0 skips the stencil)
  const int* xnz = std::is_same<T, float>::value ? nullptr : h->xnz;
  if (!S.zero_start) LAUNCH(h, K_RESIDUAL, s, launch_fine_residual<T>(h, S.b, S.x, S.r, S.part_res, s, xnz));
  // a batch decides its loop condition from all problems (enqueue_any)
  LAUNCH(h, K_INIT, s, launch_init(S.state, h->nb, S.part_res, stream_blocks(L.g), S.res_hist, S.hist_cap, cond,
                                   use_cond && h->nb == 1, s));
  enqueue_any<T>(h, S, cond, use_cond, s);
}

// Batched graphs: the loop runs while any problem of the batch runs.
template <typename T>
void enqueue_any(mg_hierarchy* h, Solver<T>& S, cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) {
  if (h->nb == 1) return;
  LAUNCH(h, K_CHECK, s, launch_any_running(S.state, h->nb, S.flag, s));
  if (use_cond) LAUNCH(h, K_CHECK, s, launch_set_cond(S.flag, cond, s));
}

template <typename T>
void enqueue_body(mg_hierarchy* h, Solver<T>& S, cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) {
  const Level& L = h->lev[h->levels - 1];
  const int C = S.C;
  if (h->opt.vcycle) {   // the multiplicative MG(V) preconditioner as the single direction
    enqueue_vcycle<T>(h, S, S.r, S.Z, S.state, s);
  } else if (h->opt.sum_columns) {   // additive MG as one preconditioner: Z = B r (Eq. 3)
    enqueue_mg<T>(h, S, S.r, S.Zmg, S.state, s);
    LAUNCH(h, K_AUX, s, launch_sum_columns<T>(L.g, S.Zmg, h->levels, S.Z, S.state, s));
  } else {
    enqueue_mg<T>(h, S, S.r, S.Z, S.state, s);
  }
  if (h->net_on) {
    if (L.g.ncomp == 3)   // the 3D vector network, one launch per layer
      LAUNCH(h, K_NET, s,
             launch_net3_forward<T>(L.g, 1, S.r, L.g.len, h->net_wtc, S.state, h->net_acts, nullptr,
                                    S.Z + (size_t)(C - 1) * L.g.cp, h->net_err, s));
    else
      LAUNCH(h, K_NET, s,
             launch_net_infer<T>(L.g, 1, S.r, L.g.len, h->net_c, h->net_wtc, S.state, nullptr,
                                 S.Z + (size_t)(C - 1) * L.g.len, h->net_err, s));
  }
  bool mf = false;
  if (h->algebraic) {
    LAUNCH(h, K_SPMM, s,
           launch_ell_spmm<T>(ell_of<T>(L.eA), S.Z + L.g.G, L.g.cp, S.AZ + L.g.G, L.g.cp, C, S.part_zaz,
                              spmm_blocks<T>(L.g, C), S.state, s));
    mf = true;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (!mf && L.kq32 && C <= 12) {   // fine operator rebuilt from the element coefficients
      LAUNCH(h, K_SPMM, s,
             launch_spmm_mf(L.g, L.kq32, S.Z, S.AZ, C, spmm_blocks<T>(L.g, C), S.part_zaz, S.state, s));
      mf = true;
    } else if (!mf && L.sth32) {   // the symmetric half of the stored stencil
      LAUNCH(h, K_SPMM, s, launch_spmm_sym(L.g, L.sth32, S.Z, S.AZ, C, S.part_zaz, S.state, s));
      mf = true;
    }
  }
  if (!mf) LAUNCH(h, K_SPMM, s, launch_spmm<T>(L.g, st_of<T>(L), S.Z, S.AZ, C, S.part_zaz, S.state, s));
  LAUNCH(h, K_GRAM, s, launch_gram_window<T>(L.g, S.win, S.Z, C, S.m, S.part_W, S.state, s));
  LAUNCH(h, K_BETA, s, launch_small_beta(S.state, h->nb, S.part_W, gram_chunks(L.g), C, S.small_scratch, S.counters,
                                         s));
  LAUNCH(h, K_ORTH, s, launch_orth_update<T>(L.g, S.win, S.Z, S.AZ, S.r, C, S.part_G, S.state, s));
  if constexpr (kIsDw<T>) LAUNCH(h, K_OGRAM, s, launch_orth_gram_dw(L.g, S.win, S.r, C, S.part_G, S.state, s));
  LAUNCH(h, K_ALPHA, s, launch_small_alpha(S.state, h->nb, S.part_G, stream_blocks(L.g), S.part_zaz,
                                          spmm_blocks<T>(L.g, C), spmm_blocks<T>(L.g, C), C, S.alpha_hist,
                                          (long long)S.hist_cap * C, S.small_scratch, S.counters, s));
  LAUNCH(h, K_UPDATE, s, launch_update_xr<T>(L.g, S.win, S.x, S.r, C, S.part_r, S.state, s));
  LAUNCH(h, K_CHECK, s, launch_check(S.state, h->nb, S.part_r, stream_blocks(L.g), S.res_hist, S.hist_cap, cond,
                                     use_cond && h->nb == 1, s));
  enqueue_any<T>(h, S, cond, use_cond, s);
}

// Capture prologue + while(cond){body} as one graph.  On any failure the
// solver falls back to direct launches with a host-side convergence test.
template <typename T>
void build_graph(mg_hierarchy* h, Solver<T>& S) {
  S.drop_graph();
  cudaGraph_t graph = nullptr;
  cudaGraphConditionalHandle cond;
  cudaStream_t cs = h->cap_stream;
  bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess;
  ok = ok && cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  ok = ok && cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                 cudaSuccess;
  if (!ok) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return;
  }
  S.prologue_launches = 0;
  h->prof.target = &S.prologue_launches;
  enqueue_prologue<T>(h, S, cond, 1, cs);
  h->prof.target = nullptr;
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  ok = cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &deps, nullptr, &ndeps) == cudaSuccess;
  ok = ok && cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp) == cudaSuccess;
  ok = ok && cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                 cudaSuccess;
  cudaGraph_t g2 = nullptr;
  const bool ended = cudaStreamEndCapture(cs, &g2) == cudaSuccess;
  ok = ok && ended;
  if (ok) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      S.body_launches = 0;
      h->prof.target = &S.body_launches;
      enqueue_body<T>(h, S, cond, 1, cs);
      h->prof.target = nullptr;
      cudaGraph_t b2 = nullptr;
      ok = cudaStreamEndCapture(cs, &b2) == cudaSuccess;
    }
  }
  cudaGraphExec_t exec = nullptr;
  ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  if (!ok) {
    cudaGraphDestroy(graph);
    cudaGetLastError();
    return;
  }
  S.graph = graph;
  S.exec = exec;
  S.use_graph = true;
}

// Run prologue + loop for solver S (buffers b, x already filled).  Returns
// per problem kd[2b] = iterations and kd[2b+1] = termination (1 converged,
// 2 maxit, 3 breakdown).
template <typename T>
mpcg_status run_solver(mg_hierarchy* h, Solver<T>& S, std::vector<int>& kd) {
  cudaStream_t s = h->stream;
  const bool direct = h->force_direct || !h->opt.use_graph;
  if (!S.use_graph && !direct) build_graph<T>(h, S);
  const bool graph = S.use_graph && !direct;
  if (graph) {
    CK(cudaGraphLaunch(S.exec, s));
  } else {
    // direct launches; the host reads the running flag after every iteration
    cudaGraphConditionalHandle dummy = 0;
    enqueue_prologue<T>(h, S, dummy, 0, s);
    for (;;) {
      int running = 0;
      if (h->nb == 1) {
        CK(cudaMemcpyAsync(&running, &S.state->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        running = running == 0;
      } else {
        CK(cudaMemcpyAsync(&running, S.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemsetAsync(S.flag, 0, sizeof(int), s));
        CK(cudaStreamSynchronize(s));
      }
      h->prof.flush();
      if (!running) break;
      enqueue_body<T>(h, S, dummy, 0, s);
    }
  }
  kd.assign(2 * (size_t)h->nb, 0);
  launch_gather_kd(S.state, h->nb, S.kdone, s);
  CK(cudaMemcpyAsync(kd.data(), S.kdone, sizeof(int) * 2 * h->nb, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (graph) {
    // the loop body ran once per x update of the slowest problem, plus once
    // more after a breakdown
    long long bodies = 0;
    for (int b = 0; b < h->nb; ++b) {
      const long long kb = kd[2 * b] + (kd[2 * b + 1] == 3 ? 1 : 0);
      if (kb > bodies) bodies = kb;
    }
    h->prof.live += S.prologue_launches + bodies * S.body_launches;
  }
  return MPCG_OK;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

mpcg_status build_f32(mg_hierarchy* h) {
  if (h->have32) return MPCG_OK;
  cudaStream_t s = h->stream;
  for (int j = 0; j < h->levels; ++j) {
    Level& L = h->lev[j];
    if (h->algebraic) {
      for (EllLevel* E : {&L.eA, &L.eP, &L.eR}) {
        if (!E->v64) continue;
        CKS(h->mem.get(&E->v32, (size_t)E->nent, s));
        launch_convert_f32(E->v64, E->v32, E->nent, s);
      }
      CKS(h->mem.get(&L.dinv32, (size_t)L.g.cp, s));
      launch_convert_f32(L.dinv64, L.dinv32, L.g.cp, s);
      continue;
    }
    CKS(h->mem.get(&L.st32, (size_t)L.nplanes * L.g.cp, s));
    CKS(h->mem.get(&L.dinv32, (size_t)L.ndinv * L.g.cp, s));
    launch_convert_f32(L.st64, L.st32, (long long)L.nplanes * L.g.cp, s);
    launch_convert_f32(L.dinv64, L.dinv32, (long long)L.ndinv * L.g.cp, s);
    if (L.g.ncomp == 1 && h->opt.half_stencil) {   // the FP32 SpMM and Jacobi stream the symmetric half
      CKS(h->mem.get(&L.sth32, (size_t)sym_planes(L.g.dim) * L.g.cp, s));
      launch_sym_half(L.g, L.st64, L.sth32, s);
    }
  }
  const GridDesc& gf = h->lev[h->levels - 1].g;
  CKS(h->mem.get(&h->b64, gf.cp, s));
  CKS(h->mem.get(&h->x64, gf.cp, s));
  CKS(h->mem.get(&h->r64, gf.cp, s));
  CKS(h->mem.get(&h->nrm, 2 * (size_t)h->nb + 2, s));
  CKS(h->mem.get(&h->part_mix, 2 * (size_t)h->nb * stream_blocks_cap(gf), s));
  CKS(h->mem.get(&h->active, h->nb, s));
  CKS(h->mem.get(&h->mix, 3 * (size_t)h->nb, s));
  CKS(h->mem.get(&h->outer, 1, s));
  CK(cudaGetLastError());
  h->have32 = true;
  return MPCG_OK;
}

// Double-word copies of the operators (MPCG_FP64_DW): stencils and sparse
// values split from the FP64 ones, inverse diagonals recomputed from them.
mpcg_status build_dw(mg_hierarchy* h) {
  if (h->havedw) return MPCG_OK;
  cudaStream_t s = h->stream;
  for (int j = 0; j < h->levels; ++j) {
    Level& L = h->lev[j];
    if (h->algebraic) {
      for (EllLevel* E : {&L.eA, &L.eP, &L.eR}) {
        if (!E->v64) continue;
        CKS(h->mem.get(&E->vdw, (size_t)E->nent, s));
        launch_convert_dw(E->v64, E->vdw, E->nent, s);
      }
      CKS(h->mem.get(&L.dinvdw, (size_t)L.g.cp, s));
      launch_convert_dw(L.dinv64, L.dinvdw, L.g.cp, s);
      continue;
    }
    CKS(h->mem.get(&L.stdw, (size_t)L.nplanes * L.g.cp, s));
    CKS(h->mem.get(&L.dinvdw, (size_t)L.ndinv * L.g.cp, s));
    launch_convert_dw(L.st64, L.stdw, (long long)L.nplanes * L.g.cp, s);
    launch_convert_dw(L.dinv64, L.dinvdw, (long long)L.ndinv * L.g.cp, s);
  }
  CK(cudaGetLastError());
  h->havedw = true;
  return MPCG_OK;
}

// Sliced ELLPACK (EllDev layout, amg::ell_layout) of a host CSR matrix,
// uploaded to the device.
mpcg_status upload_ell(mg_hierarchy* h, const mpcg::amg::Csr& M, EllLevel& E, cudaStream_t s) {
  mpcg::amg::Ell L;
  if (!mpcg::amg::ell_layout(M, L)) {
    set_err("sparse matrix too large for 32-bit entry offsets");
    return MPCG_ERR_ARG;
  }
  E.rows = L.rows;
  E.cols = L.cols;
  E.nslices = L.nslices;
  E.lg = L.lg;
  E.nent = (long long)L.col.size();
  CKS(h->mem.get(&E.sptr, L.sptr.size(), s));
  CKS(h->mem.get(&E.col, L.col.size(), s));
  CKS(h->mem.get(&E.v64, L.val.size(), s));
  if (cudaMemcpyAsync(E.sptr, L.sptr.data(), sizeof(int) * L.sptr.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(E.col, L.col.data(), sizeof(int) * L.col.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(E.v64, L.val.data(), sizeof(double) * L.val.size(), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_err("upload of a sparse operator failed: %s", cudaGetErrorString(cudaGetLastError()));
    return MPCG_ERR_CUDA;
  }
  return MPCG_OK;
}

mpcg_status check_options(const mpcg_options& opt) {
  if (opt.m < 1 || opt.m > MPCG_MAX_WINDOW || opt.nu < 1 || !(opt.omega > 0.0) || opt.pinv_tau < 0.0 ||
      opt.drop_delta < 0.0 || (opt.precision != MPCG_FP64 && opt.precision != MPCG_MIXED && opt.precision != MPCG_FP64_DW) || opt.max_outer < 1 ||
      (opt.sum_columns != 0 && opt.sum_columns != 1) || (opt.vcycle != 0 && opt.vcycle != 1) ||
      (opt.sum_columns && opt.vcycle) ||
      (opt.smoother != MPCG_SMOOTHER_JACOBI && opt.smoother != MPCG_SMOOTHER_SSOR) ||
      !(opt.ssor_omega > 0.0 && opt.ssor_omega < 2.0) || (opt.half_stencil != 0 && opt.half_stencil != 1)) {
    set_err("invalid options (m in 1..%d, nu >= 1, omega > 0, tau/delta >= 0, max_outer >= 1, sum_columns 0/1, "
            "vcycle 0/1 and not with sum_columns, smoother JACOBI/SSOR, 0 < ssor_omega < 2, half_stencil 0/1)",
            MPCG_MAX_WINDOW);
    return MPCG_ERR_ARG;
  }
  return MPCG_OK;
}

// Side streams of the MG branches, their fork/join events and the capture stream.
mpcg_status create_streams(mg_hierarchy* h) {
  bool ev_ok = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&h->ev_fine, cudaEventDisableTiming) == cudaSuccess &&
               cudaStreamCreateWithFlags(&h->side[0], cudaStreamNonBlocking) == cudaSuccess;
  for (int j = 1; j < h->levels && ev_ok; ++j)
    ev_ok = cudaStreamCreateWithFlags(&h->side[j], cudaStreamNonBlocking) == cudaSuccess;
  for (int j = 0; j < kMaxLevels && ev_ok; ++j)
    ev_ok = cudaEventCreateWithFlags(&h->ev_r[j], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&h->ev_sm[j], cudaEventDisableTiming) == cudaSuccess;
  if (!ev_ok) {
    set_err("creating streams/events failed");
    return MPCG_ERR_CUDA;
  }
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_err("cudaStreamCreateWithFlags failed");
    return MPCG_ERR_CUDA;
  }
  return MPCG_OK;
}

mpcg_status check_h(const mg_hierarchy* h) {
  if (!h) {
    set_err("hierarchy is NULL");
    return MPCG_ERR_ARG;
  }
  return MPCG_OK;
}

mpcg_status check_single(const mg_hierarchy* h) {
  CKS(check_h(h));
  if (h->nb != 1) {
    set_err("this entry point takes a single-problem hierarchy");
    return MPCG_ERR_ARG;
  }
  return MPCG_OK;
}

}  // namespace

namespace mpcg {
void set_error_message(const char* msg) { g_err = msg ? msg : ""; }
}  // namespace mpcg

extern "C" {

const char* mpcg_last_error(void) { return g_err.c_str(); }

mpcg_status mpcg_default_options(mpcg_options* opt) {
  if (!opt) {
    set_err("options pointer is NULL");
    return MPCG_ERR_ARG;
  }
  opt->m = 5;
  opt->nu = 2;
  opt->omega = 2.0 / 3.0;
  opt->pinv_tau = 1e-12;
  opt->drop_delta = 1e-10;
  opt->precision = MPCG_FP64;
  opt->inner_rtol = 3e-3;
  opt->inner_pinv_tau = 1e-6;
  opt->inner_drop_delta = 1e-5;
  opt->max_outer = 20;
  opt->use_graph = 1;
  opt->sum_columns = 0;
  opt->smoother = MPCG_SMOOTHER_JACOBI;
  opt->ssor_omega = 1.0;
  opt->vcycle = 0;
  opt->half_stencil = 1;
  opt->stream = nullptr;
  return MPCG_OK;
}

int mg_num_levels(const mg_hierarchy* h) { return h ? h->levels : -1; }
int mg_num_columns(const mg_hierarchy* h) {
  return h ? ((h->opt.sum_columns || h->opt.vcycle) ? 1 : h->levels + (h->net_on ? 1 : 0)) : -1;
}
long long mg_level_size(const mg_hierarchy* h, int level) {
  if (!h || level < 0 || level >= h->levels) return -1;
  return h->lev[level].g.n;
}

void mg_hierarchy_destroy(mg_hierarchy* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  purge_class_graphs(h->uid);
  if (h->mexec) cudaGraphExecDestroy(h->mexec);
  if (h->mgraph) cudaGraphDestroy(h->mgraph);
  h->s64.release();
  h->s32.release();
  h->sdw.release();
  h->mem.release();
  h->prof.release();
  h->net_mem.release();
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (auto sd : h->side)
    if (sd) cudaStreamDestroy(sd);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_fine) cudaEventDestroy(h->ev_fine);
  for (int j = 0; j < kMaxLevels; ++j) {
    if (h->ev_r[j]) cudaEventDestroy(h->ev_r[j]);
    if (h->ev_sm[j]) cudaEventDestroy(h->ev_sm[j]);
  }
  delete h;
}

static mpcg_status setup_impl(const mg_operator* ops, int nb, int levels, const mpcg_options* opt_in,
                              mg_hierarchy** out) {
  g_err.clear();
  if (!out) {
    set_err("out pointer is NULL");
    return MPCG_ERR_ARG;
  }
  *out = nullptr;
  if (!ops || nb < 1) {
    set_err("need at least one operator");
    return MPCG_ERR_ARG;
  }
  const mg_operator* A = ops;
  for (int b = 0; b < nb; ++b)
    if (!ops[b].values_dev || ops[b].dim != A->dim || ops[b].nodes != A->nodes || ops[b].format != A->format ||
        ops[b].dofs_per_node != A->dofs_per_node || ops[b].dirichlet_faces != A->dirichlet_faces) {
      set_err("operator %d: NULL values or a grid that differs from operator 0", b);
      return MPCG_ERR_ARG;
    }
  if (!A || !A->values_dev) {
    set_err("operator or its values pointer is NULL");
    return MPCG_ERR_ARG;
  }
  if (A->format != MPCG_FORMAT_STENCIL) {
    set_err("unsupported operator format %d", A->format);
    return MPCG_ERR_ARG;
  }
  if (A->dim != 2 && A->dim != 3) {
    set_err("dim must be 2 or 3 (got %d)", A->dim);
    return MPCG_ERR_ARG;
  }
  const int q = A->nodes - 1;   // elements per side
  if (q < 2 || q > (1 << 15)) {
    set_err("nodes - 1 must be in [2, 32768] (nodes = %d)", A->nodes);
    return MPCG_ERR_ARG;
  }
  const int ncomp = A->dofs_per_node;
  if (ncomp != 1 && !(ncomp == 3 && A->dim == 3)) {
    set_err("dofs_per_node must be 1, or 3 in 3D (got %d)", ncomp);
    return MPCG_ERR_ARG;
  }
  if (A->dirichlet_faces > MPCG_ALL_FACES) {
    set_err("dirichlet_faces 0x%x has bits beyond the six faces", A->dirichlet_faces);
    return MPCG_ERR_ARG;
  }
  const unsigned faces = A->dim == 2 ? (A->dirichlet_faces & 0xFu) : A->dirichlet_faces;   // 2D: no z faces
  // uniform coarsening halves the elements per side: nodes - 1 must be
  // divisible by 2^(levels-1), leaving at least 2 elements on the coarsest grid
  const int maxcols = ncomp > 1 ? kMaxVecCols : MPCG_MAX_COLS;
  if (levels < 1 || levels > kMaxLevels || levels > maxcols || (q % (1 << (levels - 1))) != 0 ||
      (q >> (levels - 1)) < 2) {
    set_err("levels = %d invalid for %d nodes per side (nodes - 1 must be a multiple of 2^(levels-1) with at "
            "least 2 elements per side left on the coarsest grid; at most %d levels)",
            levels, A->nodes, maxcols < kMaxLevels ? maxcols : kMaxLevels);
    return MPCG_ERR_ARG;
  }
  mpcg_options opt;
  if (opt_in) opt = *opt_in;
  else mpcg_default_options(&opt);
  CKS(check_options(opt));
  if ((opt.smoother == MPCG_SMOOTHER_SSOR || opt.vcycle) && ncomp != 1) {
    set_err("the SSOR smoother and the V-cycle are provided for scalar problems");
    return MPCG_ERR_ARG;
  }
  const long long n0 = make_grid_nodes(A->dim, (q >> (levels - 1)) + 1, faces, ncomp).n;
  if (n0 > 1024) {
    set_err("coarsest grid has %lld unknowns (> 1024); use more levels", n0);
    return MPCG_ERR_ARG;
  }
  mg_hierarchy* h = new mg_hierarchy();
  cudaGetDevice(&h->device);
  h->dim = A->dim;
  h->levels = levels;
  h->nb = nb;
  h->nodes = A->nodes;
  h->opt = opt;
  h->stream = (cudaStream_t)opt.stream;
  h->n0 = (int)n0;
  mpcg_status st = MPCG_OK;
  auto fail = [&](mpcg_status s) {
    mg_hierarchy_destroy(h);
    return s;
  };
  if ((st = create_streams(h)) != MPCG_OK) return fail(st);
  const int S = (A->dim == 3 ? 27 : 9) * ncomp;
  cudaStream_t s = h->stream;
  for (int j = 0; j < levels; ++j) {
    Level& L = h->lev[j];
    L.g = make_grid_nodes(A->dim, (q >> (levels - 1 - j)) + 1, faces, ncomp, nb);
    L.nplanes = S;
    L.ndinv = ncomp;
    if (L.g.npts >= (1LL << 31)) {
      set_err("grid too large (%lld padded entries per vector)", L.g.npts);
      return fail(MPCG_ERR_ARG);
    }
    if ((st = h->mem.get(&L.st64, (size_t)S * L.g.cp, s)) != MPCG_OK) return fail(st);
    if ((st = h->mem.get(&L.dinv64, (size_t)ncomp * L.g.cp, s)) != MPCG_OK) return fail(st);
  }
  const int J = levels - 1;
  // fine stencils: compact [S][n] per problem -> padded planes
  for (int b = 0; b < nb; ++b)
    launch_pack<double, double>(h->lev[J].g, ops[b].values_dev, h->lev[J].g.n,
                                h->lev[J].st64 + (size_t)b * h->lev[J].g.len, S, s);
  for (int j = J; j >= 1; --j) launch_galerkin(h->lev[j].g, h->lev[j - 1].g, h->lev[j].st64, h->lev[j - 1].st64, s);
  for (int j = 0; j < levels; ++j) launch_dinv<double>(h->lev[j].g, h->lev[j].st64, h->lev[j].dinv64, opt.omega, s);
  const size_t nn = (size_t)n0 * n0;
  if ((st = h->mem.get(&h->L0, nn * nb, s)) != MPCG_OK) return fail(st);
  if ((st = h->mem.get(&h->info, nb, s)) != MPCG_OK) return fail(st);
  if ((st = h->mem.get(&h->xnz, nb, s)) != MPCG_OK) return fail(st);
  {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device) == cudaSuccess) set_sm_count(nsm);
  }
  if ((st = h->mem.get(&h->rdiag0, (size_t)n0 * nb, s)) != MPCG_OK) return fail(st);
  for (int b = 0; b < nb; ++b) {
    launch_dense_from_stencil(h->lev[0].g, h->lev[0].st64 + (size_t)b * h->lev[0].g.len, h->L0 + nn * b, s);
    launch_cholesky(h->L0 + nn * b, h->rdiag0 + (size_t)n0 * b, (int)n0, h->info + b, s);
  }
  std::vector<int> info(nb, 0);
  if (cudaMemcpyAsync(info.data(), h->info, sizeof(int) * nb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_err("setup kernels failed: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(MPCG_ERR_CUDA);
  }
  for (int b = 0; b < nb; ++b)
    if (info[b] != 0) {
      set_err("coarsest operator of problem %d is not positive definite (Cholesky pivot %d)", b, info[b]);
      return fail(MPCG_ERR_NOT_SPD);
    }
  {
    double* X = nullptr;
    if ((st = h->mem.get(&h->A0inv, nn * nb, s)) != MPCG_OK) return fail(st);
    if ((st = h->mem.get(&X, nn, s)) != MPCG_OK) return fail(st);
    for (int b = 0; b < nb; ++b)
      launch_coarse_inverse(h->L0 + nn * b, h->rdiag0 + (size_t)n0 * b, X, h->A0inv + nn * b, (int)n0, s);
  }
  if ((st = build_solver<double>(h, h->s64)) != MPCG_OK) return fail(st);
  if (opt.precision == MPCG_MIXED) {
    if ((st = build_f32(h)) != MPCG_OK) return fail(st);
    if ((st = build_solver<float>(h, h->s32)) != MPCG_OK) return fail(st);
  }
  if (opt.precision == MPCG_FP64_DW) {
    if ((st = build_dw(h)) != MPCG_OK) return fail(st);
    if ((st = build_solver<dw>(h, h->sdw)) != MPCG_OK) return fail(st);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    set_err("setup failed: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(MPCG_ERR_CUDA);
  }
  *out = h;
  return MPCG_OK;
}

mpcg_status mg_hierarchy_setup(const mg_operator* A_fine, int levels, const mpcg_options* opt, mg_hierarchy** out) {
  return setup_impl(A_fine, 1, levels, opt, out);
}

mpcg_status mg_hierarchy_setup_batched(const mg_operator* ops, int nprob, int levels, const mpcg_options* opt,
                                       mg_hierarchy** out) {
  return setup_impl(ops, nprob, levels, opt, out);
}

int mg_num_problems(const mg_hierarchy* h) { return h ? h->nb : -1; }

mpcg_status mg_amg_default_options(mg_amg_options* amg) {
  if (!amg) {
    set_err("NULL options");
    return MPCG_ERR_ARG;
  }
  amg->theta = 0.4;
  amg->w = 4.0 / 3.0;
  amg->max_levels = MPCG_MAX_COLS;
  amg->coarse_size = 256;
  return MPCG_OK;
}

// Checks the matrix and the algebraic options, then builds the grids on the
// host (finest first); the coarsest grid must hold at most 1024 unknowns.
static mpcg_status amg_build_checked(const mg_csr* A, const mg_amg_options* amg_in, mpcg::amg::Levels& H) {
  if (!A) {
    set_err("matrix is NULL");
    return MPCG_ERR_ARG;
  }
  mg_amg_options amg;
  if (amg_in) amg = *amg_in;
  else mg_amg_default_options(&amg);
  if (!(amg.theta >= 0.0 && amg.theta <= 1.0) || !(amg.w >= 0.0 && amg.w <= 2.0) || amg.max_levels < 1 ||
      amg.max_levels > MPCG_MAX_COLS || amg.max_levels > kMaxLevels || amg.coarse_size < 1 ||
      amg.coarse_size > 1024) {
    set_err("invalid algebraic options (theta in [0, 1], w in [0, 2], max_levels 1..%d, coarse_size 1..1024)",
            MPCG_MAX_COLS);
    return MPCG_ERR_ARG;
  }
  if (A->n > (1 << 30)) {
    set_err("matrix: at most 2^30 rows (the flat grid pitch is a 32-bit int)");
    return MPCG_ERR_ARG;
  }
  std::string err;
  if (!mpcg::amg::check_input(A->n, A->rowptr, A->col, A->val, err)) {
    set_err("%s", err.c_str());
    return MPCG_ERR_ARG;
  }
  mpcg::amg::Csr fine;
  fine.rows = fine.cols = A->n;
  const long long nnz = A->rowptr[A->n];
  fine.ptr.assign(A->rowptr, A->rowptr + A->n + 1);
  fine.col.assign(A->col, A->col + nnz);
  fine.val.assign(A->val, A->val + nnz);
  mpcg::amg::build(fine, {amg.theta, amg.w, amg.max_levels, amg.coarse_size}, H);
  if (H.A.back().rows > 1024) {
    set_err("coarsest grid has %d unknowns (> 1024): raise max_levels or lower theta", H.A.back().rows);
    return MPCG_ERR_ARG;
  }
  return MPCG_OK;
}

mpcg_status mg_hierarchy_setup_algebraic(const mg_csr* A, const mg_amg_options* amg_in, const mpcg_options* opt_in,
                                         mg_hierarchy** out) {
  g_err.clear();
  if (!out) {
    set_err("out pointer is NULL");
    return MPCG_ERR_ARG;
  }
  *out = nullptr;
  mpcg_options opt;
  if (opt_in) opt = *opt_in;
  else mpcg_default_options(&opt);
  CKS(check_options(opt));
  if (opt.smoother != MPCG_SMOOTHER_JACOBI) {
    set_err("algebraic hierarchies smooth with damped Jacobi (the SSOR colouring needs grid coordinates)");
    return MPCG_ERR_ARG;
  }
  mpcg::amg::Levels H;
  CKS(amg_build_checked(A, amg_in, H));
  const int levels = (int)H.A.size();
  const int n0 = H.A.back().rows;
  mg_hierarchy* h = new mg_hierarchy();
  cudaGetDevice(&h->device);
  h->algebraic = true;
  h->dim = 0;
  h->levels = levels;
  h->nb = 1;
  h->nodes = 0;
  h->opt = opt;
  h->stream = (cudaStream_t)opt.stream;
  h->n0 = n0;
  mpcg_status st = MPCG_OK;
  auto fail = [&](mpcg_status e) {
    mg_hierarchy_destroy(h);
    return e;
  };
  if ((st = create_streams(h)) != MPCG_OK) return fail(st);
  {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device) == cudaSuccess) set_sm_count(nsm);
  }
  cudaStream_t s = h->stream;
  // grid j of the paper's numbering is entry levels - 1 - j of the fine-first lists
  h->amgA.resize(levels);
  h->amgP.resize(levels);
  h->amgAgg.resize(levels);
  for (int j = 0; j < levels; ++j) {
    const int l = levels - 1 - j;
    h->amgA[j] = std::move(H.A[l]);
    if (j >= 1) {
      h->amgP[j] = std::move(H.P[l]);
      h->amgAgg[j] = std::move(H.agg[l]);
    }
  }
  for (int j = 0; j < levels; ++j) {
    Level& L = h->lev[j];
    const mpcg::amg::Csr& Aj = h->amgA[j];
    L.g = make_grid_flat(Aj.rows, 1);
    L.nplanes = 0;
    L.ndinv = 1;
    if ((st = upload_ell(h, Aj, L.eA, s)) != MPCG_OK) return fail(st);
    if (j >= 1) {
      mpcg::amg::Csr Rt;
      mpcg::amg::transpose(h->amgP[j], Rt);
      if ((st = upload_ell(h, h->amgP[j], L.eP, s)) != MPCG_OK) return fail(st);
      if ((st = upload_ell(h, Rt, L.eR, s)) != MPCG_OK) return fail(st);
    }
    // damped inverse diagonal omega_j / a_ii in the flat padded layout, with
    // omega_j = min(omega, (4/3) / rho_j), rho_j the Gershgorin bound of
    // D^-1 A_j: omega_j lambda_max(D^-1 A_j) <= 4/3 keeps every level
    // correction positive definite on the wider coarse operators
    const double wj = std::min(opt.omega, (4.0 / 3.0) / mpcg::amg::gershgorin(Aj));
    std::vector<double> dv((size_t)L.g.len, 0.0);
    for (int i = 0; i < Aj.rows; ++i)
      for (int e = Aj.ptr[i]; e < Aj.ptr[i + 1]; ++e)
        if (Aj.col[e] == i) dv[(size_t)L.g.G + i] = wj / Aj.val[e];
    if ((st = h->mem.get(&L.dinv64, (size_t)L.g.cp, s)) != MPCG_OK) return fail(st);
    if (cudaMemcpyAsync(L.dinv64, dv.data(), sizeof(double) * dv.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_err("upload of the inverse diagonal failed: %s", cudaGetErrorString(cudaGetLastError()));
      return fail(MPCG_ERR_CUDA);
    }
  }
  // dense coarsest operator -> Cholesky -> inverse (as for stencil hierarchies)
  const size_t nn = (size_t)n0 * n0;
  if ((st = h->mem.get(&h->L0, nn, s)) != MPCG_OK) return fail(st);
  if ((st = h->mem.get(&h->info, 1, s)) != MPCG_OK) return fail(st);
  if ((st = h->mem.get(&h->xnz, 1, s)) != MPCG_OK) return fail(st);
  if ((st = h->mem.get(&h->rdiag0, (size_t)n0, s)) != MPCG_OK) return fail(st);
  {
    const mpcg::amg::Csr& A0 = h->amgA[0];
    std::vector<double> dense(nn, 0.0);
    for (int i = 0; i < n0; ++i)
      for (int e = A0.ptr[i]; e < A0.ptr[i + 1]; ++e) dense[(size_t)i * n0 + A0.col[e]] = A0.val[e];
    if (cudaMemcpyAsync(h->L0, dense.data(), sizeof(double) * nn, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      set_err("upload of the coarsest operator failed");
      return fail(MPCG_ERR_CUDA);
    }
    launch_cholesky(h->L0, h->rdiag0, n0, h->info, s);
    int info = 0;
    if (cudaMemcpyAsync(&info, h->info, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_err("setup kernels failed: %s", cudaGetErrorString(cudaGetLastError()));
      return fail(MPCG_ERR_CUDA);
    }
    if (info != 0) {
      set_err("coarsest operator is not positive definite (Cholesky pivot %d)", info);
      return fail(MPCG_ERR_NOT_SPD);
    }
    double* X = nullptr;
    if ((st = h->mem.get(&h->A0inv, nn, s)) != MPCG_OK) return fail(st);
    if ((st = h->mem.get(&X, nn, s)) != MPCG_OK) return fail(st);
    launch_coarse_inverse(h->L0, h->rdiag0, X, h->A0inv, n0, s);
  }
  if ((st = build_solver<double>(h, h->s64)) != MPCG_OK) return fail(st);
  if (opt.precision == MPCG_MIXED) {
    if ((st = build_f32(h)) != MPCG_OK) return fail(st);
    if ((st = build_solver<float>(h, h->s32)) != MPCG_OK) return fail(st);
  }
  if (opt.precision == MPCG_FP64_DW) {
    if ((st = build_dw(h)) != MPCG_OK) return fail(st);
    if ((st = build_solver<dw>(h, h->sdw)) != MPCG_OK) return fail(st);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    set_err("setup failed: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(MPCG_ERR_CUDA);
  }
  *out = h;
  return MPCG_OK;
}

static const mpcg::amg::Csr* amg_matrix(const mg_hierarchy* h, int level, int which) {
  if (!h || !h->algebraic || level < 0 || level >= h->levels) return nullptr;
  if (which == MPCG_AMG_A) return &h->amgA[level];
  if (which == MPCG_AMG_P && level >= 1) return &h->amgP[level];
  return nullptr;
}

mpcg_status mg_amg_aggregates(const mg_hierarchy* h, int level, int* agg) {
  g_err.clear();
  if (!h || !h->algebraic || level < 1 || level >= h->levels || !agg) {
    set_err("need an algebraic hierarchy, a grid level >= 1 and an output array");
    return MPCG_ERR_ARG;
  }
  const std::vector<int>& a = h->amgAgg[level];
  std::copy(a.begin(), a.end(), agg);
  return MPCG_OK;
}

long long mg_amg_nnz(const mg_hierarchy* h, int level, int which) {
  const mpcg::amg::Csr* M = amg_matrix(h, level, which);
  return M ? M->nnz() : -1;
}

mpcg_status mg_amg_get(const mg_hierarchy* h, int level, int which, int* rowptr, int* col, double* val) {
  g_err.clear();
  const mpcg::amg::Csr* M = amg_matrix(h, level, which);
  if (!M || !rowptr || !col || !val) {
    set_err("need an algebraic hierarchy, a valid level/matrix and output arrays");
    return MPCG_ERR_ARG;
  }
  std::copy(M->ptr.begin(), M->ptr.end(), rowptr);
  std::copy(M->col.begin(), M->col.end(), col);
  std::copy(M->val.begin(), M->val.end(), val);
  return MPCG_OK;
}

}  // extern "C"

// Host-only hierarchy: the grids of the paper's numbering (0 coarsest).
struct mg_amg_host {
  std::vector<mpcg::amg::Csr> A, P;
  std::vector<std::vector<int>> agg;
};

extern "C" {

mpcg_status mg_amg_setup_host(const mg_csr* A, const mg_amg_options* amg, mg_amg_host** out) {
  g_err.clear();
  if (!out) {
    set_err("out pointer is NULL");
    return MPCG_ERR_ARG;
  }
  *out = nullptr;
  mpcg::amg::Levels H;
  CKS(amg_build_checked(A, amg, H));
  const int levels = (int)H.A.size();
  mg_amg_host* a = new mg_amg_host();
  a->A.resize(levels);
  a->P.resize(levels);
  a->agg.resize(levels);
  for (int j = 0; j < levels; ++j) {
    const int l = levels - 1 - j;
    a->A[j] = std::move(H.A[l]);
    if (j >= 1) {
      a->P[j] = std::move(H.P[l]);
      a->agg[j] = std::move(H.agg[l]);
    }
  }
  *out = a;
  return MPCG_OK;
}

int mg_amg_host_levels(const mg_amg_host* a) { return a ? (int)a->A.size() : -1; }

long long mg_amg_host_size(const mg_amg_host* a, int level) {
  if (!a || level < 0 || level >= (int)a->A.size()) return -1;
  return a->A[level].rows;
}

static const mpcg::amg::Csr* host_matrix(const mg_amg_host* a, int level, int which) {
  if (!a || level < 0 || level >= (int)a->A.size()) return nullptr;
  if (which == MPCG_AMG_A) return &a->A[level];
  if (which == MPCG_AMG_P && level >= 1) return &a->P[level];
  return nullptr;
}

long long mg_amg_host_nnz(const mg_amg_host* a, int level, int which) {
  const mpcg::amg::Csr* M = host_matrix(a, level, which);
  return M ? M->nnz() : -1;
}

mpcg_status mg_amg_host_aggregates(const mg_amg_host* a, int level, int* agg) {
  g_err.clear();
  if (!a || level < 1 || level >= (int)a->A.size() || !agg) {
    set_err("need a host hierarchy, a grid level >= 1 and an output array");
    return MPCG_ERR_ARG;
  }
  std::copy(a->agg[level].begin(), a->agg[level].end(), agg);
  return MPCG_OK;
}

mpcg_status mg_amg_host_get(const mg_amg_host* a, int level, int which, int* rowptr, int* col, double* val) {
  g_err.clear();
  const mpcg::amg::Csr* M = host_matrix(a, level, which);
  if (!M || !rowptr || !col || !val) {
    set_err("need a host hierarchy, a valid level/matrix and output arrays");
    return MPCG_ERR_ARG;
  }
  std::copy(M->ptr.begin(), M->ptr.end(), rowptr);
  std::copy(M->col.begin(), M->col.end(), col);
  std::copy(M->val.begin(), M->val.end(), val);
  return MPCG_OK;
}

static bool host_ell(const mg_amg_host* a, int level, int which, mpcg::amg::Ell& E) {
  mpcg::amg::Csr Rt;
  const mpcg::amg::Csr* M = nullptr;
  if (which == MPCG_AMG_R) {
    const mpcg::amg::Csr* P = host_matrix(a, level, MPCG_AMG_P);
    if (!P) return false;
    mpcg::amg::transpose(*P, Rt);
    M = &Rt;
  } else {
    M = host_matrix(a, level, which);
  }
  return M && mpcg::amg::ell_layout(*M, E);
}

long long mg_amg_host_ell_entries(const mg_amg_host* a, int level, int which) {
  mpcg::amg::Ell E;
  return host_ell(a, level, which, E) ? (long long)E.col.size() : -1;
}

mpcg_status mg_amg_host_ell(const mg_amg_host* a, int level, int which, int* lg, int* nslices, int* sptr, int* col,
                            double* val) {
  g_err.clear();
  mpcg::amg::Ell E;
  if (!lg || !nslices || !sptr || !col || !val || !host_ell(a, level, which, E)) {
    set_err("need a host hierarchy, a valid level/matrix and output arrays");
    return MPCG_ERR_ARG;
  }
  *lg = E.lg;
  *nslices = E.nslices;
  std::copy(E.sptr.begin(), E.sptr.end(), sptr);
  std::copy(E.col.begin(), E.col.end(), col);
  std::copy(E.val.begin(), E.val.end(), val);
  return MPCG_OK;
}

void mg_amg_host_destroy(mg_amg_host* a) { delete a; }

}  // extern "C"

// The FP64-data solve: T = double (FP64 arithmetic) or dw (double-word
// arithmetic on the FP32 pipe; b and x0 are split into pairs on entry and x
// is assembled back into doubles).
template <typename T>
static mpcg_status solve_fp64(mg_hierarchy* h, Solver<T>& S, const double* b, double* x, double rtol, int maxit,
                              int* iters_out, double* res_hist, double* alpha_hist) {
  cudaStream_t s = h->stream;
  const GridDesc& gf = h->lev[h->levels - 1].g;
  const int nb = h->nb;
  CKS(ensure_hist(h, S, maxit));
  for (int p = 0; p < nb; ++p) {
    LAUNCH(h, K_PACK, s, launch_pack<double, T>(gf, b + (size_t)p * gf.n, gf.n, S.b + (size_t)p * gf.len, 1, s));
    CK(cudaMemsetAsync(h->xnz + p, 0, sizeof(int), s));
    LAUNCH(h, K_PACK, s, launch_pack_flag<T>(gf, x + (size_t)p * gf.n, S.x + (size_t)p * gf.len, h->xnz + p, s));
  }
  LAUNCH(h, K_AUX, s, launch_set_params(S.state, nb, rtol, maxit, S.m, S.C, h->opt.drop_delta, h->opt.pinv_tau, s));
  std::vector<int> kd;
  CKS(run_solver<T>(h, S, kd));
  for (int p = 0; p < nb; ++p) {
    LAUNCH(h, K_PACK, s, launch_unpack<T, double>(gf, S.x + (size_t)p * gf.len, x + (size_t)p * gf.n, gf.n, 1, s));
    const int k = kd[2 * p];
    if (res_hist)
      CK(cudaMemcpyAsync(res_hist + (size_t)p * (maxit + 1), S.res_hist + (size_t)p * S.hist_cap,
                         sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, s));
    if (alpha_hist && k > 0)
      CK(cudaMemcpyAsync(alpha_hist + (size_t)p * maxit * S.C, S.alpha_hist + (size_t)p * S.hist_cap * S.C,
                         sizeof(double) * k * S.C, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  mpcg_status result = MPCG_OK;
  for (int p = 0; p < nb; ++p) {
    if (iters_out) iters_out[p] = kd[2 * p];
    if (kd[2 * p + 1] == 3) {
      set_err("breakdown in problem %d at iteration %d (non-finite value or every column dropped)", p, kd[2 * p]);
      result = MPCG_ERR_BREAKDOWN;
    } else if (kd[2 * p + 1] != 1 && result == MPCG_OK) {
      result = MPCG_NOT_CONVERGED;
    }
  }
  return result;
}

extern "C" {

// The mixed-precision solve as one CUDA graph: an outer conditional while
// node (FP64 residual, device-side decision, scaling, FP32 inner solve,
// FP64 update) whose body holds the inner solver's prologue and its own
// conditional while node.  No host round trip per refinement step.
static void drop_mixed_graph(mg_hierarchy* h) {
  if (h->mexec) cudaGraphExecDestroy(h->mexec);
  if (h->mgraph) cudaGraphDestroy(h->mgraph);
  h->mexec = nullptr;
  h->mgraph = nullptr;
  h->mg_rtol = -1.0;
  h->mg_maxit = h->mg_hist = -1;
  ++h->graph_gen;
}

static cudaGraphNode_t add_while(cudaStream_t cs, cudaGraph_t g, cudaGraphConditionalHandle c, cudaGraph_t* body,
                                 bool* ok) {
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = c;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  *ok = *ok && cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &deps, nullptr, &ndeps) == cudaSuccess;
  *ok = *ok && cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp) == cudaSuccess;
  *ok = *ok && cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                   cudaSuccess;
  if (*ok) *body = cp.conditional.phGraph_out[0];
  return node;
}

// Capture h's whole mixed-precision solve (init, the refinement while node
// and its body with the inner while node) into `graph` as a new root branch.
// Several hierarchies captured into one graph run concurrently in one launch.
static bool capture_mixed(mg_hierarchy* h, cudaGraph_t graph, double rtol, int maxit) {
  Solver<float>& S = h->s32;
  const int J = h->levels - 1;
  const Level& L = h->lev[J];
  const GridDesc& gf = L.g;
  const int nb = h->nb;
  cudaStream_t cs = h->cap_stream;
  cudaGraph_t obody = nullptr, ibody = nullptr;
  cudaGraphConditionalHandle c_out, c_in;
  bool ok = cudaGraphConditionalHandleCreate(&c_out, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  ok = ok && cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                 cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return false;
  }
  long long init_launches = 0;   // the one init launch is counted per solve by the caller
  h->prof.target = &init_launches;
  LAUNCH(h, K_AUX, cs, launch_mix_init(h->mix, h->active, nb, h->outer, cs));
  add_while(cs, graph, c_out, &obody, &ok);
  cudaGraph_t tmp = nullptr;
  ok = (cudaStreamEndCapture(cs, &tmp) == cudaSuccess) && ok;
  // outer body: residual, decision, scaling, inner solve, update
  ok = ok && cudaStreamBeginCaptureToGraph(cs, obody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                 cudaSuccess;
  if (ok) {
    h->mg_head = 0;
    h->prof.target = &h->mg_head;
    LAUNCH(h, K_RESIDUAL, cs, launch_fine_residual<double>(h, h->b64, h->x64, h->r64, h->part_mix, cs, h->xnz));
    LAUNCH(h, K_AUX, cs, launch_sum_partials(h->part_mix, nb, 2, stream_blocks(gf), h->nrm, cs));
    LAUNCH(h, K_AUX, cs, launch_outer_check(h->mix, h->active, nb, h->nrm, rtol, maxit, h->opt.max_outer, h->outer,
                                            S.state, h->opt.inner_rtol, S.m, S.C, h->opt.inner_drop_delta,
                                            h->opt.inner_pinv_tau, c_out, cs));
    LAUNCH(h, K_AUX, cs, launch_start_inner(gf, h->r64, h->nrm, h->active, S.b, S.r, S.part_res, cs));
    ok = cudaMemsetAsync(S.x, 0, sizeof(float) * gf.cp, cs) == cudaSuccess;
    ok = ok && cudaGraphConditionalHandleCreate(&c_in, obody, 0, 0) == cudaSuccess;
    if (ok) {
      h->mg_iprol = 0;
      h->prof.target = &h->mg_iprol;
      enqueue_prologue<float>(h, S, c_in, 1, cs);
      add_while(cs, obody, c_in, &ibody, &ok);
      h->mg_tail = 0;
      h->prof.target = &h->mg_tail;
      LAUNCH(h, K_AUX, cs, launch_outer_accumulate(h->mix, nb, S.state, cs));
      LAUNCH(h, K_AUX, cs, launch_axpy_mixed(gf, h->x64, S.x, h->nrm, h->xnz, cs));
    }
    h->prof.target = nullptr;
    ok = (cudaStreamEndCapture(cs, &tmp) == cudaSuccess) && ok;
  }
  // inner body: one MPCG iteration
  ok = ok && cudaStreamBeginCaptureToGraph(cs, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                 cudaSuccess;
  if (ok) {
    h->mg_ibody = 0;
    h->prof.target = &h->mg_ibody;
    enqueue_body<float>(h, S, c_in, 1, cs);
    h->prof.target = nullptr;
    ok = (cudaStreamEndCapture(cs, &tmp) == cudaSuccess) && ok;
  }
  h->prof.target = nullptr;
  if (!ok) cudaGetLastError();
  return ok;
}

static bool build_mixed_graph(mg_hierarchy* h, double rtol, int maxit) {
  drop_mixed_graph(h);
  cudaGraph_t graph = nullptr;
  bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess;
  ok = ok && capture_mixed(h, graph, rtol, maxit);
  cudaGraphExec_t exec = nullptr;
  ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  if (!ok) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return false;
  }
  h->mgraph = graph;
  h->mexec = exec;
  h->mg_rtol = rtol;
  h->mg_maxit = maxit;
  h->mg_hist = h->s32.hist_cap;
  return true;
}

namespace {
void drop_mixed_graph_fwd(mg_hierarchy* h) { drop_mixed_graph(h); }
}  // namespace

// The graph form of solve_mixed (no histories).  Returns MPCG_ERR_CUDA with
// *fallback = true when the graph cannot be built (the caller then runs the
// host-driven loop).
static mpcg_status solve_mixed_graph(mg_hierarchy* h, const double* b, double* x, double rtol, int maxit,
                                     int* iters_out, bool* fallback) {
  *fallback = false;
  CKS(build_f32(h));
  CKS(build_solver<float>(h, h->s32));
  Solver<float>& S = h->s32;
  CKS(ensure_hist(h, S, maxit));
  cudaStream_t s = h->stream;
  const GridDesc& gf = h->lev[h->levels - 1].g;
  const int nb = h->nb;
  if (!h->mexec || h->mg_rtol != rtol || h->mg_maxit != maxit || h->mg_hist != S.hist_cap) {
    if (!build_mixed_graph(h, rtol, maxit)) {
      *fallback = true;
      return MPCG_ERR_CUDA;
    }
  }
  for (int p = 0; p < nb; ++p) {
    LAUNCH(h, K_PACK, s, launch_pack<double, double>(gf, b + (size_t)p * gf.n, gf.n, h->b64 + (size_t)p * gf.len, 1, s));
    CK(cudaMemsetAsync(h->xnz + p, 0, sizeof(int), s));
    LAUNCH(h, K_PACK, s, launch_pack_flag(gf, x + (size_t)p * gf.n, h->x64 + (size_t)p * gf.len, h->xnz + p, s));
  }
  CK(cudaGraphLaunch(h->mexec, s));
  for (int p = 0; p < nb; ++p)
    LAUNCH(h, K_PACK, s, launch_unpack<double, double>(gf, h->x64 + (size_t)p * gf.len, x + (size_t)p * gf.n, gf.n, 1, s));
  std::vector<int> mix(3 * (size_t)nb);
  int steps = 0;
  CK(cudaMemcpyAsync(mix.data(), h->mix, sizeof(int) * 3 * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&steps, h->outer, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  // launches executed: init, per step the head, inner prologue and tail, per
  // inner iteration the body (the slowest problem's count for a batch)
  long long kmax = 0;
  for (int p = 0; p < nb; ++p) kmax = std::max<long long>(kmax, mix[3 * p]);
  h->prof.live += 1 + (long long)steps * (h->mg_head + h->mg_iprol + h->mg_tail) + kmax * h->mg_ibody;
  mpcg_status result = MPCG_OK;
  for (int p = 0; p < nb; ++p) {
    if (iters_out) iters_out[p] = mix[3 * p];
    const int status = mix[3 * p + 1];
    if (status == 3) {
      set_err("breakdown in the FP32 inner solve of problem %d", p);
      result = MPCG_ERR_BREAKDOWN;
    } else if (status != 1 && result == MPCG_OK) {
      result = MPCG_NOT_CONVERGED;
    }
  }
  return result;
}

// Whether mpcg_solve_batched_graph takes these classes: mixed precision,
// graphs enabled, one device, no hierarchy twice.
static bool classes_graph_eligible(mg_hierarchy* const* hs, int nclass) {
  if (!hs || nclass < 1) return false;
  for (int c = 0; c < nclass; ++c) {
    const mg_hierarchy* h = hs[c];
    if (!h || h->opt.precision != MPCG_MIXED || !h->opt.use_graph || h->force_direct || h->device != hs[0]->device)
      return false;
    for (int d = 0; d < c; ++d)
      if (hs[d] == h) return false;
  }
  return true;
}

mpcg_status mpcg_solve_batched_graph(mg_hierarchy* const* hs, int nclass, const double* const* b,
                                     double* const* x, double rtol, int maxit, int* const* iters) {
  g_err.clear();
  if (!hs || nclass < 1 || !b || !x) {
    set_err("mpcg_solve_batched_graph: bad arguments");
    return MPCG_ERR_ARG;
  }
  if (maxit < 0 || !(rtol >= 0.0)) {
    set_err("maxit must be >= 0 and rtol >= 0");
    return MPCG_ERR_ARG;
  }
  for (int c = 0; c < nclass; ++c) {
    CKS(check_h(hs[c]));
    if (!b[c] || !x[c]) {
      set_err("b[%d] and x[%d] must not be NULL", c, c);
      return MPCG_ERR_ARG;
    }
  }
  if (!classes_graph_eligible(hs, nclass)) {
    set_err("mpcg_solve_batched_graph: every class must be a distinct mixed-precision hierarchy with graphs "
            "enabled, all on one device");
    return MPCG_ERR_ARG;
  }
  CK(cudaSetDevice(hs[0]->device));
  cudaStream_t s = hs[0]->stream;
  for (int c = 0; c < nclass; ++c) {
    mg_hierarchy* h = hs[c];
    CKS(build_f32(h));
    CKS(build_solver<float>(h, h->s32));
    CKS(ensure_hist(h, h->s32, maxit));
    if (h->stream != s) CK(cudaStreamSynchronize(h->stream));   // earlier work on the class's own stream
  }
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_class_graph_mu);
    for (auto& e : g_class_graphs) {
      bool same = e.rtol == rtol && e.maxit == maxit && (int)e.uid.size() == nclass;
      for (int c = 0; same && c < nclass; ++c)
        same = e.uid[c] == hs[c]->uid && e.gen[c] == hs[c]->graph_gen && e.hist[c] == hs[c]->s32.hist_cap;
      if (same) {
        exec = e.exec;
        break;
      }
    }
  }
  if (!exec) {
    ClassGraph e;
    e.rtol = rtol;
    e.maxit = maxit;
    bool ok = cudaGraphCreate(&e.graph, 0) == cudaSuccess;
    for (int c = 0; c < nclass && ok; ++c) ok = capture_mixed(hs[c], e.graph, rtol, maxit);
    ok = ok && cudaGraphInstantiate(&e.exec, e.graph, 0) == cudaSuccess;
    if (!ok) {
      destroy_class_graph(e);
      cudaGetLastError();
      set_err("mpcg_solve_batched_graph: the graph of the classes could not be built");
      return MPCG_ERR_CUDA;
    }
    for (int c = 0; c < nclass; ++c) {
      e.uid.push_back(hs[c]->uid);
      e.gen.push_back(hs[c]->graph_gen);
      e.hist.push_back(hs[c]->s32.hist_cap);
    }
    exec = e.exec;
    std::lock_guard<std::mutex> lk(g_class_graph_mu);
    if (g_class_graphs.size() >= kMaxClassGraphs) {
      destroy_class_graph(g_class_graphs.front());
      g_class_graphs.erase(g_class_graphs.begin());
    }
    g_class_graphs.push_back(e);
  }
  // inputs: pack every class's b and x0 (host arrays staged as in mpcg_solve)
  std::vector<const double*> bd(nclass);
  std::vector<double*> xd(nclass);
  std::vector<char> xhost(nclass, 0);
  for (int c = 0; c < nclass; ++c) {
    mg_hierarchy* h = hs[c];
    const GridDesc& gf = h->lev[h->levels - 1].g;
    const size_t ntot = (size_t)gf.n * h->nb;
    bd[c] = b[c];
    xd[c] = x[c];
    const bool bdev = is_device_pointer(b[c]), xdev = is_device_pointer(x[c]);
    if (!bdev || !xdev) {
      if (!h->stage) CKS(h->mem.get(&h->stage, 2 * ntot, s));
      if (!bdev) {
        CK(cudaMemcpyAsync(h->stage, b[c], sizeof(double) * ntot, cudaMemcpyHostToDevice, s));
        bd[c] = h->stage;
      }
      if (!xdev) {
        CK(cudaMemcpyAsync(h->stage + ntot, x[c], sizeof(double) * ntot, cudaMemcpyHostToDevice, s));
        xd[c] = h->stage + ntot;
        xhost[c] = 1;
      }
    }
    h->prof.reset();
    if (h->net_on && h->net_err) CK(cudaMemsetAsync(h->net_err, 0, sizeof(int), s));
    for (int p = 0; p < h->nb; ++p) {
      LAUNCH(h, K_PACK, s, launch_pack<double, double>(gf, bd[c] + (size_t)p * gf.n, gf.n,
                                                        h->b64 + (size_t)p * gf.len, 1, s));
      CK(cudaMemsetAsync(h->xnz + p, 0, sizeof(int), s));
      LAUNCH(h, K_PACK, s, launch_pack_flag(gf, xd[c] + (size_t)p * gf.n, h->x64 + (size_t)p * gf.len, h->xnz + p, s));
    }
  }
  CK(cudaGraphLaunch(exec, s));
  std::vector<std::vector<int>> mix(nclass);
  std::vector<int> steps(nclass, 0), nerr(nclass, 0);
  for (int c = 0; c < nclass; ++c) {
    mg_hierarchy* h = hs[c];
    const GridDesc& gf = h->lev[h->levels - 1].g;
    for (int p = 0; p < h->nb; ++p)
      LAUNCH(h, K_PACK, s, launch_unpack<double, double>(gf, h->x64 + (size_t)p * gf.len, xd[c] + (size_t)p * gf.n,
                                                          gf.n, 1, s));
    mix[c].resize(3 * (size_t)h->nb);
    CK(cudaMemcpyAsync(mix[c].data(), h->mix, sizeof(int) * 3 * h->nb, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&steps[c], h->outer, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (h->net_on && h->net_err) CK(cudaMemcpyAsync(&nerr[c], h->net_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  mpcg_status worst = MPCG_OK;
  std::string msg;
  for (int c = 0; c < nclass; ++c) {
    mg_hierarchy* h = hs[c];
    const GridDesc& gf = h->lev[h->levels - 1].g;
    long long kmax = 0;
    for (int p = 0; p < h->nb; ++p) kmax = std::max<long long>(kmax, mix[c][3 * p]);
    h->prof.live += 1 + (long long)steps[c] * (h->mg_head + h->mg_iprol + h->mg_tail) + kmax * h->mg_ibody;
    h->prof.flush();
    h->last_launches = h->prof.live;
    mpcg_status st = MPCG_OK;
    std::string cmsg;
    for (int p = 0; p < h->nb; ++p) {
      if (iters && iters[c]) iters[c][p] = mix[c][3 * p];
      const int status = mix[c][3 * p + 1];
      if (status == 3) {
        if (st != MPCG_ERR_BREAKDOWN) cmsg = "breakdown in the FP32 inner solve of problem " + std::to_string(p);
        st = MPCG_ERR_BREAKDOWN;
      } else if (status != 1 && st == MPCG_OK) {
        st = MPCG_NOT_CONVERGED;
      }
    }
    if (nerr[c]) {
      st = MPCG_ERR_TIMEOUT;
      cmsg = "learned column: a tensor-core wait timed out";
    }
    if (xhost[c] && (st >= 0 || st == MPCG_ERR_BREAKDOWN))
      CK(cudaMemcpyAsync(x[c], xd[c], sizeof(double) * (size_t)gf.n * h->nb, cudaMemcpyDeviceToHost, s));
    if (st < 0 && (worst >= 0 || st < worst)) {
      worst = st;
      msg = "class " + std::to_string(c) + ": " + cmsg;
    } else if (st == MPCG_NOT_CONVERGED && worst == MPCG_OK) {
      worst = st;
      msg = "class " + std::to_string(c) + " did not converge";
    }
  }
  CK(cudaStreamSynchronize(s));
  if (worst != MPCG_OK) set_err("%s", msg.c_str());
  return worst;
}

static mpcg_status solve_mixed(mg_hierarchy* h, const double* b, double* x, double rtol, int maxit, int* iters_out,
                               double* res_hist) {
  CKS(build_f32(h));
  CKS(build_solver<float>(h, h->s32));
  Solver<float>& S = h->s32;
  cudaStream_t s = h->stream;
  const Level& L = h->lev[h->levels - 1];
  const GridDesc& gf = L.g;
  CKS(ensure_hist(h, S, maxit));
  const int nb = h->nb;
  for (int p = 0; p < nb; ++p) {
    LAUNCH(h, K_PACK, s, launch_pack<double, double>(gf, b + (size_t)p * gf.n, gf.n, h->b64 + (size_t)p * gf.len, 1, s));
    CK(cudaMemsetAsync(h->xnz + p, 0, sizeof(int), s));
    LAUNCH(h, K_PACK, s, launch_pack_flag(gf, x + (size_t)p * gf.n, h->x64 + (size_t)p * gf.len, h->xnz + p, s));
  }
  // every problem refines on its own true FP64 residual; the problems run
  // their FP32 inner solves together, converged ones with a zero right-hand
  // side (their inner solve stops at once)
  std::vector<int> total(nb, 0), nhist(nb, 0), status(nb, 0), act(nb, 1);
  std::vector<double> nrm(2 * (size_t)nb), inner(maxit + 1);
  for (int outer = 0; outer <= h->opt.max_outer; ++outer) {
    LAUNCH(h, K_RESIDUAL, s, launch_fine_residual<double>(h, h->b64, h->x64, h->r64, h->part_mix, s, h->xnz));
    LAUNCH(h, K_AUX, s, launch_sum_partials(h->part_mix, nb, 2, stream_blocks(gf), h->nrm, s));
    CK(cudaMemcpyAsync(nrm.data(), h->nrm, 2 * sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int running = 0, budget = 0;
    for (int p = 0; p < nb; ++p) {
      if (!act[p]) continue;
      const double rn = sqrt(nrm[2 * p]), bn = sqrt(nrm[2 * p + 1]);
      double* rh = res_hist ? res_hist + (size_t)p * (maxit + 1) : nullptr;
      if (outer == 0 && rh) rh[nhist[p]++] = bn > 0 ? rn / bn : 0.0;
      if (!isfinite(rn)) {
        status[p] = 3;
        act[p] = 0;
      } else if (bn == 0.0 || rn <= rtol * bn) {
        status[p] = 1;
        act[p] = 0;
      } else if (total[p] >= maxit || outer == h->opt.max_outer) {
        status[p] = 2;
        act[p] = 0;
      } else {
        ++running;
        budget = std::max(budget, maxit - total[p]);
      }
    }
    if (!running) break;
    CK(cudaMemcpyAsync(h->active, act.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s));
    LAUNCH(h, K_AUX, s, launch_start_inner(gf, h->r64, h->nrm, h->active, S.b, S.r, S.part_res, s));
    CK(cudaMemsetAsync(S.x, 0, sizeof(float) * gf.cp, s));
    LAUNCH(h, K_AUX, s, launch_set_params(S.state, nb, h->opt.inner_rtol, budget, S.m, S.C, h->opt.inner_drop_delta,
                                          h->opt.inner_pinv_tau, s));
    std::vector<int> kd;
    CKS(run_solver<float>(h, S, kd));
    for (int p = 0; p < nb; ++p) {
      if (!act[p]) continue;
      const int k = kd[2 * p];
      if (res_hist && k > 0) {
        double* rh = res_hist + (size_t)p * (maxit + 1);
        const double rn = sqrt(nrm[2 * p]), bn = sqrt(nrm[2 * p + 1]);
        CK(cudaMemcpyAsync(inner.data(), S.res_hist + (size_t)p * S.hist_cap, sizeof(double) * (k + 1),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int i = 1; i <= k && nhist[p] <= maxit; ++i) rh[nhist[p]++] = inner[i] * rn / bn;
      }
      total[p] += k;
      if (kd[2 * p + 1] == 3) {
        status[p] = 3;
        act[p] = 0;
      } else if (k == 0) {
        status[p] = 2;
        act[p] = 0;
      }
    }
    LAUNCH(h, K_AUX, s, launch_axpy_mixed(gf, h->x64, S.x, h->nrm, h->xnz, s));
  }
  for (int p = 0; p < nb; ++p)
    LAUNCH(h, K_PACK, s, launch_unpack<double, double>(gf, h->x64 + (size_t)p * gf.len, x + (size_t)p * gf.n, gf.n, 1, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  mpcg_status result = MPCG_OK;
  for (int p = 0; p < nb; ++p) {
    if (iters_out) iters_out[p] = total[p];
    if (status[p] == 3) {
      set_err("breakdown in the FP32 inner solve of problem %d", p);
      result = MPCG_ERR_BREAKDOWN;
    } else if (status[p] != 1 && result == MPCG_OK) {
      result = MPCG_NOT_CONVERGED;
    }
  }
  return result;
}

mpcg_status mpcg_solve(mg_hierarchy* h, const double* b, double* x, double rtol, int maxit, int* iters_out,
                       double* res_hist, double* alpha_hist) {
  g_err.clear();
  CKS(check_h(h));
  if (!b || !x) {
    set_err("b and x must not be NULL");
    return MPCG_ERR_ARG;
  }
  if (maxit < 0 || !(rtol >= 0.0)) {
    set_err("maxit must be >= 0 and rtol >= 0");
    return MPCG_ERR_ARG;
  }
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  const GridDesc& gf = h->lev[h->levels - 1].g;
  const size_t ntot = (size_t)gf.n * h->nb;   // unknowns of all problems of the batch
  const size_t nb = sizeof(double) * ntot;
  const bool bdev = is_device_pointer(b), xdev = is_device_pointer(x);
  const double* bd = b;
  double* xd = x;
  if (!bdev || !xdev) {
    if (!h->stage) CKS(h->mem.get(&h->stage, 2 * ntot, s));
    if (!bdev) {
      CK(cudaMemcpyAsync(h->stage, b, nb, cudaMemcpyHostToDevice, s));
      bd = h->stage;
    }
    if (!xdev) {
      CK(cudaMemcpyAsync(h->stage + ntot, x, nb, cudaMemcpyHostToDevice, s));
      xd = h->stage + ntot;
    }
  }
  h->prof.reset();
  if (h->net_on && h->net_err) CK(cudaMemsetAsync(h->net_err, 0, sizeof(int), s));
  mpcg_status st;
  if (h->opt.precision == MPCG_MIXED) {
    bool fallback = true;
    st = MPCG_OK;
    if (h->opt.use_graph && !h->force_direct && !res_hist) st = solve_mixed_graph(h, bd, xd, rtol, maxit, iters_out, &fallback);
    if (fallback) st = solve_mixed(h, bd, xd, rtol, maxit, iters_out, res_hist);
  } else if (h->opt.precision == MPCG_FP64_DW) {
    st = solve_fp64<dw>(h, h->sdw, bd, xd, rtol, maxit, iters_out, res_hist, alpha_hist);
  } else {
    st = solve_fp64<double>(h, h->s64, bd, xd, rtol, maxit, iters_out, res_hist, alpha_hist);
  }
  h->prof.flush();
  h->last_launches = h->prof.live;
  if (h->net_on && h->net_err) {
    int err = 0;
    CK(cudaMemcpyAsync(&err, h->net_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (err) {
      set_err("learned column: a tensor-core wait timed out");
      st = MPCG_ERR_TIMEOUT;
    }
  }
  if (!xdev && (st >= 0 || st == MPCG_ERR_BREAKDOWN)) {
    CK(cudaMemcpyAsync(x, xd, nb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return st;
}

// ---------------------------------------------------------------------------
// Autotuner: launch shapes timed per kernel class on this hierarchy's grids
// and arithmetic (see tune.h for the table and its JSON cache).

static void drop_all_graphs(mg_hierarchy* h) {
  cudaStreamSynchronize(h->stream);
  h->s64.drop_graph();
  h->s32.drop_graph();
  h->sdw.drop_graph();
  drop_mixed_graph(h);
}

mpcg_status mg_autotune(mg_hierarchy* h, const char* cache_path, int* timed_out) {
  g_err.clear();
  CKS(check_h(h));
  if (timed_out) *timed_out = 0;
  CK(cudaSetDevice(h->device));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, h->device));
  const int sms = prop.multiProcessorCount;
  const int J = h->levels - 1;
  const GridDesc gf = h->lev[J].g;
  const int nb = h->nb;
  const int prec = h->opt.precision;
  const int kind = prec == MPCG_MIXED ? tune::kF32 : (prec == MPCG_FP64_DW ? tune::kDW : tune::kF64);
  const int C = prec == MPCG_MIXED ? h->s32.C : (prec == MPCG_FP64_DW ? h->sdw.C : h->s64.C);
  struct Tunable {
    int fn, kind;
    long long npts;
    int C, dflt, lo, hi;
    std::vector<int> metric;   // kernel classes the shape acts on (documentation)
  };
  std::vector<Tunable> keys;
  keys.push_back({tune::kStream, tune::kAny, gf.npts, 0, stream_blocks_default(gf), stream_blocks_min(gf),
                  stream_blocks_cap(gf), {K_ORTH, K_UPDATE, K_RESIDUAL, K_INIT, K_CHECK}});
  keys.push_back({tune::kGram, tune::kAny, gf.npts, 0, gram_chunks_default(gf), gram_chunks_min(gf),
                  gram_chunks_cap(gf), {K_GRAM, K_BETA}});
  {
    int d = 0;
    if (kind == tune::kF32) d = spmm_blocks<float>(gf, C);
    else if (kind == tune::kDW) d = spmm_blocks<dw>(gf, C);
    else d = spmm_blocks<double>(gf, C);
    keys.push_back({tune::kSpmm, kind, gf.npts, C, d, stream_blocks_min(gf), stream_blocks_cap(gf), {K_SPMM, K_ALPHA}});
  }
  if (!h->algebraic && h->opt.smoother == MPCG_SMOOTHER_JACOBI)
    for (int j = 1; j <= J; ++j) {
      const GridDesc& g = h->lev[j].g;
      if (g.ncomp != 1) continue;
      const bool rule = g.npts / (kind == tune::kF32 ? 4 : 2) * g.nb < (long long)sms * 128;
      keys.push_back({tune::kJacobi, kind, g.npts, 0, rule ? 1 : 0, 0, 1, {K_JACOBI}});
    }
  // a cache written on this device that holds every key: no timing
  if (cache_path && tune::load(cache_path, prop.name, sms) >= 0) {
    bool all = true;
    for (const Tunable& k : keys) {
      int v;
      all = all && tune::find(k.fn, k.kind, k.npts, nb, k.C, &v);
    }
    if (all) {
      drop_all_graphs(h);
      return MPCG_OK;
    }
  }
  // time the candidates on profiled solves of a fixed right-hand side
  Alloc mem;
  cudaStream_t s = h->stream;
  double *b = nullptr, *x = nullptr;
  const size_t n = (size_t)gf.n * nb;
  mpcg_status st = mem.get(&b, n, s);
  if (st == MPCG_OK) st = mem.get(&x, n, s);
  if (st != MPCG_OK) {
    mem.release();
    return st;
  }
  {
    std::vector<double> hb(n);
    unsigned long long z = 0x2545F4914F6CDD1DULL;
    for (size_t i = 0; i < n; ++i) {   // splitmix64 -> uniform in [-1, 1)
      z += 0x9E3779B97F4A7C15ULL;
      unsigned long long t = z;
      t = (t ^ (t >> 30)) * 0xBF58476D1CE4E5B9ULL;
      t = (t ^ (t >> 27)) * 0x94D049BB133111EBULL;
      t ^= t >> 31;
      hb[i] = (double)(t >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
    if (cudaMemcpyAsync(b, hb.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      mem.release();
      set_err("mg_autotune: upload of the right-hand side failed");
      return MPCG_ERR_CUDA;
    }
  }
  int timed = 0;
  // the objective is the whole solve as it runs (graph launch, concurrent
  // multigrid branches): per-kernel times of a serialised profiled solve
  // miss how the branches overlap.  Best of three batches of five solves.
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    mem.release();
    set_err("mg_autotune: cudaEventCreate failed");
    return MPCG_ERR_CUDA;
  }
  auto measure = [&](const Tunable& k, double* out) -> mpcg_status {
    (void)k;
    drop_all_graphs(h);
    double best = 1e300;
    for (int rep = 0; rep < 4; ++rep) {
      if (cudaEventRecord(e0, s) != cudaSuccess) return MPCG_ERR_CUDA;
      for (int i = 0; i < 5; ++i) {
        if (cudaMemsetAsync(x, 0, sizeof(double) * n, s) != cudaSuccess) return MPCG_ERR_CUDA;
        int it = 0;
        const mpcg_status r = mpcg_solve(h, b, x, 1e-8, 500, &it, nullptr, nullptr);
        if (r != MPCG_OK && r != MPCG_NOT_CONVERGED) return r;
      }
      float ms = 0.f;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        return MPCG_ERR_CUDA;
      if (rep > 0 && ms < best) best = ms;   // the first batch rebuilds the graph and warms up
    }
    ++timed;
    *out = best;
    return MPCG_OK;
  };
  for (const Tunable& k : keys) {
    std::vector<int> cand = {k.dflt};
    if (k.fn == tune::kJacobi) {
      cand = {0, 1};
    } else if (k.fn == tune::kGram) {
      for (int f : {k.dflt / 2, 2 * k.dflt, 4 * k.dflt}) cand.push_back(f);
    } else {
      for (int f : {1, 2, 3, 4, 6, 8}) cand.push_back(f * sms);
    }
    int cur = k.dflt;
    if (tune::find(k.fn, k.kind, k.npts, nb, k.C, &cur) && cur >= k.lo && cur <= k.hi) cand.insert(cand.begin(), cur);
    int best_v = k.dflt;
    double best_t = 1e300;
    std::vector<int> seen;
    for (int v : cand) {
      if (v < k.lo || v > k.hi || std::find(seen.begin(), seen.end(), v) != seen.end()) continue;
      seen.push_back(v);
      tune::set(k.fn, k.kind, k.npts, nb, k.C, v);
      double t = 0.0;
      st = measure(k, &t);
      if (st != MPCG_OK) break;
      if (t < best_t) {
        best_t = t;
        best_v = v;
      }
    }
    tune::set(k.fn, k.kind, k.npts, nb, k.C, best_v);
    if (st != MPCG_OK) break;
  }
  drop_all_graphs(h);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  mem.release();
  if (timed_out) *timed_out = timed;
  if (st != MPCG_OK) {
    set_err("mg_autotune: a timed solve failed: %s", g_err.c_str());
    return st;
  }
  if (cache_path && !tune::save(cache_path, prop.name, sms)) {
    set_err("mg_autotune: cannot write the cache file %s", cache_path);
    return MPCG_ERR_ARG;
  }
  return MPCG_OK;
}

mpcg_status mg_autotune_load(const char* cache_path, const char* device_name, int sm_count, int* entries) {
  g_err.clear();
  if (!cache_path || !device_name) {
    set_err("mg_autotune_load: NULL path or device name");
    return MPCG_ERR_ARG;
  }
  const int r = tune::load(cache_path, device_name, sm_count);
  if (r < 0) {
    set_err(r == -1 ? "mg_autotune_load: no such file" : r == -2 ? "mg_autotune_load: malformed cache file"
                                                               : "mg_autotune_load: cache written for another device");
    return MPCG_ERR_ARG;
  }
  if (entries) *entries = r;
  return MPCG_OK;
}

mpcg_status mg_autotune_save(const char* cache_path, const char* device_name, int sm_count) {
  g_err.clear();
  if (!cache_path || !device_name || !tune::save(cache_path, device_name, sm_count)) {
    set_err("mg_autotune_save: cannot write the cache file");
    return MPCG_ERR_ARG;
  }
  return MPCG_OK;
}

int mg_autotune_lookup(int tunable, int kind, long long npts, int nb, int ncols) {
  int v = -1;
  return tune::find(tunable, kind, npts, nb, ncols, &v) ? v : -1;
}

void mg_autotune_set(int tunable, int kind, long long npts, int nb, int ncols, int value) {
  if (tunable >= 0 && tunable < tune::kNumTunables) tune::set(tunable, kind, npts, nb, ncols, value);
}

void mg_autotune_clear(void) { tune::clear(); }

const char* mpcg_kernel_class_name(int cls) {
  return cls >= 0 && cls < K_COUNT ? kClassNames[cls] : "";
}

long long mg_last_launches(const mg_hierarchy* h) { return h ? h->last_launches : -1; }

mpcg_status mg_last_solve_counters(const mg_hierarchy* h, int problem, int* out4) {
  g_err.clear();
  if (!h || !out4 || problem < 0 || problem >= h->nb) {
    set_err("mg_last_solve_counters: NULL argument or problem index out of range");
    return MPCG_ERR_ARG;
  }
  const DevState* st = h->opt.precision == MPCG_MIXED    ? h->s32.state
                        : h->opt.precision == MPCG_FP64_DW ? h->sdw.state
                                                           : h->s64.state;
  if (!st) {
    out4[0] = out4[1] = out4[2] = out4[3] = 0;
    return MPCG_OK;
  }
  CK(cudaSetDevice(h->device));
  DevState d;
  CK(cudaMemcpyAsync(&d, st + problem, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  out4[0] = d.k;
  out4[1] = d.done;
  out4[2] = d.dropped_total;
  out4[3] = d.pinv_fallbacks;
  return MPCG_OK;
}

mpcg_status mpcg_solve_profiled(mg_hierarchy* h, const double* b, double* x, double rtol, int maxit, int* iters_out,
                                double* class_ms, long long* class_launches, int* trace_cls, float* trace_ms,
                                long long trace_cap, long long* trace_len) {
  CKS(check_h(h));
  h->prof.on = true;
  h->force_direct = true;
  mpcg_status st = mpcg_solve(h, b, x, rtol, maxit, iters_out, nullptr, nullptr);
  h->prof.on = false;
  h->force_direct = false;
  for (int i = 0; i < K_COUNT; ++i) {
    if (class_ms) class_ms[i] = h->prof.ms[i];
    if (class_launches) class_launches[i] = h->prof.count[i];
  }
  const long long nt = (long long)h->prof.trace.size();
  if (trace_len) *trace_len = nt;
  for (long long i = 0; i < nt && i < trace_cap; ++i) {
    if (trace_cls) trace_cls[i] = h->prof.trace[i].first;
    if (trace_ms) trace_ms[i] = h->prof.trace[i].second;
  }
  return st;
}

mpcg_status mg_apply_operator(mg_hierarchy* h, int level, const double* X, double* Y, int ncols) {
  g_err.clear();
  CKS(check_single(h));
  if (level < 0 || level >= h->levels || ncols < 1 || !X || !Y) {
    set_err("bad level, column count or pointer");
    return MPCG_ERR_ARG;
  }
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  const Level& L = h->lev[level];
  double *xp = nullptr, *yp = nullptr;
  const int maxc = L.g.ncomp > 1 ? kMaxVecCols : kMaxCols;
  const int chunk = ncols < maxc ? ncols : maxc;
  CK(cudaMalloc(&xp, sizeof(double) * chunk * L.g.len));
  CK(cudaMalloc(&yp, sizeof(double) * chunk * L.g.len));
  cudaMemsetAsync(xp, 0, sizeof(double) * chunk * L.g.len, s);
  for (int c0 = 0; c0 < ncols; c0 += chunk) {
    const int nc = ncols - c0 < chunk ? ncols - c0 : chunk;
    launch_pack<double, double>(L.g, X + (size_t)c0 * L.g.n, L.g.n, xp, nc, s);
    if (h->algebraic)
      launch_ell_spmm<double>(ell_of<double>(L.eA), xp + L.g.G, L.g.len, yp + L.g.G, L.g.len, nc, nullptr, 0, nullptr,
                              s);
    else
      launch_spmm<double>(L.g, L.st64, xp, yp, nc, nullptr, nullptr, s);
    launch_unpack<double, double>(L.g, yp, Y + (size_t)c0 * L.g.n, L.g.n, nc, s);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(xp);
  cudaFree(yp);
  CK(e);
  CK(cudaGetLastError());
  return MPCG_OK;
}

mpcg_status mg_corrections(mg_hierarchy* h, const double* r, double* Z) {
  g_err.clear();
  CKS(check_single(h));
  if (!r || !Z) {
    set_err("NULL pointer");
    return MPCG_ERR_ARG;
  }
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  Solver<double>& S = h->s64;
  const GridDesc& gf = h->lev[h->levels - 1].g;
  launch_pack<double, double>(gf, r, gf.n, S.r, 1, s);
  if (h->opt.vcycle) {   // one column: the V-cycle B_V r
    enqueue_vcycle<double>(h, S, S.r, S.Z, nullptr, s);
    launch_unpack<double, double>(gf, S.Z, Z, gf.n, 1, s);
  } else {
    double* Zc = h->opt.sum_columns ? S.Zmg : S.Z;   // the per-grid columns
    enqueue_mg<double>(h, S, S.r, Zc, nullptr, s);
    launch_unpack<double, double>(gf, Zc, Z, gf.n, h->levels, s);
  }
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  return MPCG_OK;
}

mpcg_status mg_apply_operator_f32(mg_hierarchy* h, int level, const double* X, double* Y, int ncols) {
  g_err.clear();
  CKS(check_single(h));
  if (level < 0 || level >= h->levels || ncols < 1 || !X || !Y) {
    set_err("bad level, column count or pointer");
    return MPCG_ERR_ARG;
  }
  if (h->algebraic || h->opt.precision != MPCG_MIXED) {
    set_err("the FP32 operators exist on stencil hierarchies built with precision MPCG_MIXED");
    return MPCG_ERR_ARG;
  }
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  const Level& L = h->lev[level];
  float *xp = nullptr, *yp = nullptr;
  const int maxc = L.g.ncomp > 1 ? kMaxVecCols : kMaxCols;
  const int chunk = ncols < maxc ? ncols : maxc;
  CK(cudaMalloc(&xp, sizeof(float) * chunk * L.g.len));
  CK(cudaMalloc(&yp, sizeof(float) * chunk * L.g.len));
  cudaMemsetAsync(xp, 0, sizeof(float) * chunk * L.g.len, s);
  for (int c0 = 0; c0 < ncols; c0 += chunk) {
    const int nc = ncols - c0 < chunk ? ncols - c0 : chunk;
    launch_pack<double, float>(L.g, X + (size_t)c0 * L.g.n, L.g.n, xp, nc, s);
    if (L.sth32) launch_spmm_sym(L.g, L.sth32, xp, yp, nc, nullptr, nullptr, s);
    else launch_spmm<float>(L.g, L.st32, xp, yp, nc, nullptr, nullptr, s);
    launch_unpack<float, double>(L.g, yp, Y + (size_t)c0 * L.g.n, L.g.n, nc, s);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(xp);
  cudaFree(yp);
  CK(e);
  CK(cudaGetLastError());
  return MPCG_OK;
}

mpcg_status mg_corrections_f32(mg_hierarchy* h, const double* r, double* Z) {
  g_err.clear();
  CKS(check_single(h));
  if (!r || !Z) {
    set_err("NULL pointer");
    return MPCG_ERR_ARG;
  }
  if (h->algebraic || h->opt.precision != MPCG_MIXED) {
    set_err("the FP32 operators exist on stencil hierarchies built with precision MPCG_MIXED");
    return MPCG_ERR_ARG;
  }
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  Solver<float>& S = h->s32;
  const GridDesc& gf = h->lev[h->levels - 1].g;
  launch_pack<double, float>(gf, r, gf.n, S.r, 1, s);
  if (h->opt.vcycle) {
    enqueue_vcycle<float>(h, S, S.r, S.Z, nullptr, s);
    launch_unpack<float, double>(gf, S.Z, Z, gf.n, 1, s);
  } else {
    float* Zc = h->opt.sum_columns ? S.Zmg : S.Z;
    enqueue_mg<float>(h, S, S.r, Zc, nullptr, s);
    launch_unpack<float, double>(gf, Zc, Z, gf.n, h->levels, s);
  }
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  return MPCG_OK;
}

mpcg_status mg_get_operator(mg_hierarchy* h, int level, double* planes) {
  g_err.clear();
  CKS(check_single(h));
  if (level < 0 || level >= h->levels || !planes) {
    set_err("bad level or pointer");
    return MPCG_ERR_ARG;
  }
  if (h->algebraic) {
    set_err("an algebraic hierarchy has no stencil planes (mg_amg_get returns its matrices)");
    return MPCG_ERR_ARG;
  }
  CK(cudaSetDevice(h->device));
  const Level& L = h->lev[level];
  launch_unpack<double, double>(L.g, L.st64, planes, L.g.n, L.nplanes, h->stream);
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaGetLastError());
  return MPCG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned search column (an extension beyond the paper).
namespace {

// the 3x3x3 network of 3D vector problems, else the 3x3 one of 2D problems
bool net3_of(const mg_hierarchy* h) {
  const GridDesc& g = h->lev[h->levels - 1].g;
  return h->dim == 3 && g.ncomp == 3 && h->nb == 1 && !h->algebraic;
}
int net_params_of(const mg_hierarchy* h) { return net3_of(h) ? kNet3Params : kNetParams; }

mpcg_status net_check_grid(const mg_hierarchy* h) {
  const GridDesc& g = h->lev[h->levels - 1].g;
  if (net3_of(h)) return MPCG_OK;
  if (h->dim != 2 || h->nb != 1 || g.ncomp != 1 || g.nx != g.ny || g.px != g.py || g.lp < 0) {
    set_err("the learned column is implemented for single (unbatched) scalar 2D problems with Dirichlet faces "
            "and for single 3D vector problems (3 unknowns per node)");
    return MPCG_ERR_ARG;
  }
  return MPCG_OK;
}

// Coefficient channel and inference buffers of hierarchy h.
mpcg_status net_prepare(mg_hierarchy* h) {
  if (h->net_wq) return MPCG_OK;
  cudaStream_t s = h->stream;
  const Level& L = h->lev[h->levels - 1];
  if (net3_of(h)) {   // the 3D network: activations on the node box, no coefficient channel
    const size_t alen = (size_t)net3_act_len(L.g);
    CKS(h->net_mem.get(&h->net_wq, kNet3Params, s));
    CKS(h->net_mem.get(&h->net_acts.a0, alen * 16, s));
    CKS(h->net_mem.get(&h->net_acts.a1, alen * 16, s));
    CKS(h->net_mem.get(&h->net_acts.a2, alen * 16, s));
    CKS(h->net_mem.get(&h->net_acts.a3, alen * 16, s));
    CKS(h->net_mem.get(&h->net_err, 1, s));
    CKS(h->net_mem.get(&h->net_wtc, (size_t)net3_pack_bytes(), s));
    net3_prepare_attributes();
    CK(cudaGetLastError());
    return MPCG_OK;
  }
  double* part = nullptr;
  CKS(h->net_mem.get(&h->net_c, L.g.len, s));
  CKS(h->net_mem.get(&part, 256, s));
  CKS(h->net_mem.get(&h->net_wq, kNetParams, s));
  CKS(h->net_mem.get(&h->net_acts.a0, (size_t)L.g.len * kNetIn, s));
  CKS(h->net_mem.get(&h->net_acts.a1, (size_t)L.g.len * kNetC1, s));
  CKS(h->net_mem.get(&h->net_acts.a2, (size_t)L.g.len * kNetW, s));
  CKS(h->net_mem.get(&h->net_acts.a3, (size_t)L.g.len * kNetW, s));
  CKS(h->net_mem.get(&h->net_err, 1, s));
  CKS(h->net_mem.get(&h->net_wtc, (size_t)net_tc_weight_bytes(), s));
  net_infer_prepare_attributes();
  launch_net_coef(L.g, L.dinv64, h->opt.omega, h->net_c, part, s);
  CK(cudaGetLastError());
  return MPCG_OK;
}

// Copy n floats from host or device memory into device memory.
mpcg_status copy_floats(float* dst, const float* src, int n, cudaStream_t s) {
  CK(cudaMemcpyAsync(dst, src, sizeof(float) * n, is_device_pointer(src) ? cudaMemcpyDeviceToDevice
                                                                         : cudaMemcpyHostToDevice, s));
  return MPCG_OK;
}

// Buffers of one training batch of up to B images on grid g: inputs, A e,
// the network's outputs and activations, the data gradients, the
// weight-gradient partials (2D: the 3x3 network; net3: the 3x3x3 one).
struct NetBatch {
  bool net3 = false;
  int np = 0;
  float *rb = nullptr, *eb = nullptr, *aeb = nullptr, *y = nullptr, *ay = nullptr, *dy = nullptr, *d4 = nullptr;
  double *dots = nullptr, *coef = nullptr;
  NetActs a = {};
  NetGrads gr = {};
  unsigned char* wtc = nullptr;
  int* terr = nullptr;
  double** parts_dev = nullptr;
};

int net_batch_blocks(const NetBatch& nb, const GridDesc& g, int nimg) {
  return nb.net3 ? net3_wgrad_blocks(g, nimg) : net_wgrad_tc_blocks(g, nimg);
}

mpcg_status net_batch_alloc(bool net3, const GridDesc& g, int B, Alloc& mem, cudaStream_t s, NetBatch& nb) {
  nb.net3 = net3;
  nb.np = net3 ? kNet3Params : kNetParams;
  mpcg_status st = MPCG_OK;
  auto get = [&](auto** p, size_t n) {
    if (st == MPCG_OK) st = mem.get(p, n, s);
  };
  const size_t L = g.len;
  const size_t A = net3 ? (size_t)net3_act_len(g) : L;   // points of one activation image
  const int nw = net_batch_blocks(nb, g, B);
  get(&nb.rb, B * L);
  get(&nb.eb, B * L);
  get(&nb.aeb, B * L);
  get(&nb.y, B * L);
  get(&nb.ay, B * L);
  get(&nb.dy, B * L);
  get(&nb.a.a0, B * A * (net3 ? 16 : kNetIn));
  get(&nb.a.a1, B * A * 16);
  get(&nb.a.a2, B * A * 16);
  get(&nb.a.a3, B * A * 16);
  get(&nb.gr.d1, B * A * 16);
  get(&nb.gr.d2, B * A * 16);
  get(&nb.gr.d3, B * A * 16);
  if (net3) get(&nb.d4, B * A * 16);
  const size_t lsz[4] = {net3 ? 16 * 3 * 27u : (size_t)kNetC1 * kNetIn * 9, net3 ? 16 * 16 * 27u : (size_t)kNetW * kNetC1 * 9,
                         net3 ? 16 * 16 * 27u : (size_t)kNetW * kNetW * 9, net3 ? 3 * 16 * 27u : (size_t)kNetW * 9};
  for (int l = 0; l < 4; ++l) get(&nb.gr.part[l], lsz[l] * nw);
  get(&nb.dots, 3 * 64 * B);
  get(&nb.coef, 2 * B);
  get(&nb.wtc, (size_t)(net3 ? net3_pack_bytes() : net_tc_weight_bytes()));
  get(&nb.terr, 1);
  get(&nb.parts_dev, 4);
  if (st != MPCG_OK) return st;
  if (net3) net3_prepare_attributes();
  else net_train_tc_prepare_attributes();
  CK(cudaMemcpyAsync(nb.parts_dev, nb.gr.part, sizeof(nb.gr.part), cudaMemcpyHostToDevice, s));
  return MPCG_OK;
}

// One forward and backward pass on nimg images already in nb.rb / eb / aeb:
// y, A y, the loss (added to loss_sum), dL/dy and the weight-gradient
// partials.  c: the 2D network's coefficient channel; st32: the FP32 fine
// operator.
void net_batch_step(NetBatch& nb, const GridDesc& g, int nimg, const float* c, const float* st32, const float* wq,
                    double* loss_sum, cudaStream_t s) {
  if (nb.net3) {
    launch_net3_pack(wq, nb.wtc, s);
    launch_net3_forward<float>(g, nimg, nb.rb, g.len, nb.wtc, nullptr, nb.a, nb.y, (float*)nullptr, nb.terr, s);
  } else {
    launch_net_pack_tc(wq, nb.wtc, s);
    launch_net_infer<float>(g, nimg, nb.rb, g.len, c, nb.wtc, nullptr, nb.y, (float*)nullptr, nb.terr, s, nullptr,
                            nb.a);
  }
  launch_spmm<float>(g, st32, nb.y, nb.ay, nimg, nullptr, nullptr, s);
  launch_net_loss_grad(g, nimg, nb.y, nb.ay, nb.eb, nb.aeb, nb.dots, nb.coef, loss_sum, nb.dy, s);
  if (nb.net3) launch_net3_backward(g, nimg, nb.wtc, nb.a, nb.dy, nb.gr, nb.d4, nb.terr, s);
  else launch_net_backward(g, nimg, wq, nb.a, nb.dy, nb.gr, nb.terr, s);
}

// Rebuild the solvers after the column count changed.
void drop_mixed_graph_fwd(mg_hierarchy* h);
mpcg_status rebuild_solvers(mg_hierarchy* h) {
  CK(cudaStreamSynchronize(h->stream));
  drop_mixed_graph_fwd(h);
  const bool had32 = h->s32.built, haddw = h->sdw.built;
  h->s64.release();
  h->s32.release();
  h->sdw.release();
  CKS(build_solver<double>(h, h->s64));
  if (had32) CKS(build_solver<float>(h, h->s32));
  if (haddw) CKS(build_solver<dw>(h, h->sdw));
  return MPCG_OK;
}

}  // namespace

extern "C" {

int mg_learned_num_params(void) { return kNetParams; }

int mg_learned_num_params_of(const mg_hierarchy* h) { return h ? net_params_of(h) : -1; }

mpcg_status mg_set_tensor_wait_limit(long long polls) {
  g_err.clear();
  if (polls < 0) {
    set_err("polls must be >= 0");
    return MPCG_ERR_ARG;
  }
  CK(set_wait_first_infer(polls));
  CK(set_wait_first_train(polls));
  CK(set_wait_first_net3(polls));
  return MPCG_OK;
}

mpcg_status mg_learned_attach(mg_hierarchy* h, const float* params, int nparams) {
  g_err.clear();
  CKS(check_h(h));
  CKS(net_check_grid(h));
  const int np = net_params_of(h);
  if (!params || nparams != np) {
    set_err("params must hold mg_learned_num_params_of(h) = %d floats", np);
    return MPCG_ERR_ARG;
  }
  if (h->levels + 1 > (net3_of(h) ? kMaxVecCols : MPCG_MAX_COLS) || h->opt.sum_columns || h->opt.vcycle) {
    set_err("too many grids for an extra column, or the columns are summed into one / a V-cycle");
    return MPCG_ERR_ARG;
  }
  CK(cudaSetDevice(h->device));
  CKS(net_prepare(h));
  float* tmp = nullptr;
  CK(cudaMalloc(&tmp, sizeof(float) * np));
  mpcg_status st = copy_floats(tmp, params, np, h->stream);
  if (st == MPCG_OK) {
    launch_round_bf16(tmp, h->net_wq, np, h->stream);
    if (net3_of(h)) launch_net3_pack(h->net_wq, h->net_wtc, h->stream);
    else launch_net_pack_tc(h->net_wq, h->net_wtc, h->stream);
  }
  cudaStreamSynchronize(h->stream);
  cudaFree(tmp);
  if (st != MPCG_OK) return st;
  CK(cudaGetLastError());
  if (!h->net_on) {
    h->net_on = true;
    CKS(rebuild_solvers(h));
  }
  return MPCG_OK;
}

mpcg_status mg_learned_detach(mg_hierarchy* h) {
  g_err.clear();
  CKS(check_h(h));
  CK(cudaSetDevice(h->device));
  if (h->net_on) {
    h->net_on = false;
    CKS(rebuild_solvers(h));
  }
  return MPCG_OK;
}

mpcg_status mg_attach_q1_kappa(mg_hierarchy* h, const double* kappa_dev) {
  g_err.clear();
  CKS(check_h(h));
  Level& L = h->lev[h->levels - 1];
  if (!kappa_dev || L.g.ncomp != 1 || h->algebraic) {
    set_err("mg_attach_q1_kappa: scalar stencil hierarchies and a device kappa array only");
    return MPCG_ERR_ARG;
  }
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  CKS(build_f32(h));
  const int nodes = h->nodes;   // elements per side: nodes - 1
  if (!L.kq32_store) CKS(h->mem.get(&L.kq32_store, L.g.cp, s));
  double* k64 = nullptr;
  unsigned long long* chk = nullptr;
  if (cudaMalloc(&k64, sizeof(double) * L.g.cp) != cudaSuccess ||
      cudaMalloc(&chk, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(k64);
    cudaGetLastError();
    set_err("mg_attach_q1_kappa: device allocation failed");
    return MPCG_ERR_OOM;
  }
  double dmax = 0.0, amax = 0.0;
  mpcg_status st = MPCG_OK;
  if (cudaMemsetAsync(k64, 0, sizeof(double) * L.g.cp, s) != cudaSuccess ||
      cudaMemsetAsync(L.kq32_store, 0, sizeof(float) * L.g.cp, s) != cudaSuccess)
    st = MPCG_ERR_CUDA;
  if (st == MPCG_OK)
    st = place_kappa(L.g, kappa_dev, nodes - 1, 1.0 / (nodes - 1), L.kq32_store, k64, chk, L.st64, &dmax, &amax, s);
  cudaFree(k64);
  cudaFree(chk);
  // the slots were rewritten: until the check passes, the stored operator is in use
  L.kq32 = nullptr;
  h->s32.drop_graph();
  drop_mixed_graph_fwd(h);
  CKS(st);
  CK(cudaGetLastError());
  if (!(dmax <= 1e-10 * amax)) {
    set_err("mg_attach_q1_kappa: the stored fine operator is not the Q1 diffusion operator of this kappa "
            "(largest coefficient difference %.3e of %.3e)", dmax, amax);
    return MPCG_ERR_ARG;
  }
  L.kq32 = L.kq32_store;
  return MPCG_OK;
}

mpcg_status mg_detach_q1_kappa(mg_hierarchy* h) {
  g_err.clear();
  CKS(check_h(h));
  h->lev[h->levels - 1].kq32 = nullptr;
  h->s32.drop_graph();
  drop_mixed_graph_fwd(h);
  return MPCG_OK;
}

mpcg_status mg_learned_forward_acts(mg_hierarchy* h, const float* rhat_dev, float* y_dev, float* acts_dev,
                                   int nimg) {
  g_err.clear();
  CKS(check_h(h));
  CKS(net_check_grid(h));
  if (!h->net_on || !rhat_dev || !y_dev || nimg < 1) {
    set_err("attach weights first; rhat, y must be device arrays of nimg >= 1 images");
    return MPCG_ERR_ARG;
  }
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  const GridDesc& g = h->lev[h->levels - 1].g;
  Alloc tmp;
  float *r = nullptr, *y = nullptr;
  mpcg_status st = MPCG_OK;
  NetActs a3 = {};
  if (net3_of(h)) {   // activations for nimg images
    const size_t A = (size_t)net3_act_len(g) * nimg * 16;
    for (__nv_bfloat16** p : {&a3.a0, &a3.a1, &a3.a2, &a3.a3})
      if (st == MPCG_OK) st = tmp.get(p, A, s);
  }
  if (st == MPCG_OK && (st = tmp.get(&r, (size_t)nimg * g.len, s)) == MPCG_OK &&
      (st = tmp.get(&y, (size_t)nimg * g.len, s)) == MPCG_OK) {
    cudaMemsetAsync(h->net_err, 0, sizeof(int), s);
    launch_pack<float, float>(g, rhat_dev, g.n, r, nimg, s);
    if (net3_of(h)) {
      launch_net3_forward<float>(g, nimg, r, g.len, h->net_wtc, nullptr, a3, y, (float*)nullptr, h->net_err, s);
      if (acts_dev) launch_net3_acts_export(g, nimg, a3, acts_dev, s);
    } else {
      launch_net_infer<float>(g, nimg, r, g.len, h->net_c, h->net_wtc, nullptr, y, (float*)nullptr, h->net_err, s,
                              acts_dev);
    }
    launch_unpack<float, float>(g, y, y_dev, g.n, nimg, s);
    int err = 0;
    if (cudaMemcpyAsync(&err, h->net_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      set_err("learned forward failed");
      st = MPCG_ERR_CUDA;
    } else if (err) {
      set_err("learned forward: a tensor-core wait timed out");
      st = MPCG_ERR_TIMEOUT;
    }
  }
  tmp.release();
  return st;
}

mpcg_status mg_learned_forward(mg_hierarchy* h, const float* rhat_dev, float* y_dev, int nimg) {
  return mg_learned_forward_acts(h, rhat_dev, y_dev, nullptr, nimg);
}

mpcg_status mg_learned_grad(mg_hierarchy* h, const float* params, const float* rhat_dev, const float* e_dev,
                            int nimg, double* grad, float* acts_dev, float* y_dev, double* loss) {
  g_err.clear();
  CKS(check_h(h));
  CKS(net_check_grid(h));
  const bool net3 = net3_of(h);
  const int maxb = net3 ? kMaxVecCols : MPCG_MAX_COLS;
  if (!params || !rhat_dev || !e_dev || !grad || nimg < 1 || nimg > maxb) {
    set_err("mg_learned_grad: params, rhat, e and grad are required and nimg must be in 1..%d", maxb);
    return MPCG_ERR_ARG;
  }
  CK(cudaSetDevice(h->device));
  cudaStream_t s = h->stream;
  const GridDesc g = h->lev[h->levels - 1].g;
  if (!net3 && g.p > 1024) {
    set_err("training grids are limited to 1025 nodes per side");
    return MPCG_ERR_ARG;
  }
  CKS(build_f32(h));
  CKS(net_prepare(h));
  Alloc mem;
  NetBatch nbt;
  mpcg_status st = net_batch_alloc(net3, g, nimg, mem, s, nbt);
  double *lsum = nullptr, *gd = nullptr;
  float *master = nullptr, *wq = nullptr;
  if (st == MPCG_OK) st = mem.get(&lsum, 1, s);
  if (st == MPCG_OK) st = mem.get(&gd, nbt.np, s);
  if (st == MPCG_OK) st = mem.get(&master, nbt.np, s);
  if (st == MPCG_OK) st = mem.get(&wq, nbt.np, s);
  if (st != MPCG_OK) {
    mem.release();
    return st;
  }
  copy_floats(master, params, nbt.np, s);
  launch_round_bf16(master, wq, nbt.np, s);
  launch_pack<float, float>(g, rhat_dev, g.n, nbt.rb, nimg, s);
  launch_pack<float, float>(g, e_dev, g.n, nbt.eb, nimg, s);
  const float* st32 = h->lev[h->levels - 1].st32;
  launch_spmm<float>(g, st32, nbt.eb, nbt.aeb, nimg, nullptr, nullptr, s);
  cudaMemsetAsync(lsum, 0, sizeof(double), s);
  net_batch_step(nbt, g, nimg, h->net_c, st32, wq, lsum, s);
  launch_net_grad_sum(nbt.parts_dev, net_batch_blocks(nbt, g, nimg), net3 ? 1 : 0, gd, s);
  if (acts_dev) {
    if (net3) launch_net3_acts_export(g, nimg, nbt.a, acts_dev, s);
    else launch_net_acts_export(g, nimg, nbt.a, acts_dev, s);
  }
  if (y_dev) launch_unpack<float, float>(g, nbt.y, y_dev, g.n, nimg, s);
  double lh = 0.0;
  int terr_h = 0;
  if (cudaMemcpyAsync(grad, gd, sizeof(double) * nbt.np,
                      is_device_pointer(grad) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&lh, lsum, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&terr_h, nbt.terr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    set_err("mg_learned_grad: %s", cudaGetErrorString(cudaGetLastError()));
    st = MPCG_ERR_CUDA;
  } else if (terr_h) {
    set_err("mg_learned_grad: a tensor-core wait timed out");
    st = MPCG_ERR_TIMEOUT;
  }
  if (loss) *loss = lh;
  mem.release();
  return st;
}

mpcg_status mg_learned_train(mg_hierarchy* const* hs, int nprob, const int* pair_prob, int npairs,
                             const float* rhat_dev, const float* e_dev, const mg_train_opts* opts, float* params,
                             double* loss_hist) {
  g_err.clear();
  if (!hs || nprob < 1 || !pair_prob || npairs < 1 || !rhat_dev || !e_dev || !opts || !params) {
    set_err("mg_learned_train: bad arguments");
    return MPCG_ERR_ARG;
  }
  CKS(check_h(hs[0]));
  const bool net3 = net3_of(hs[0]);
  const int B = opts->batch;
  const int maxb = net3 ? kMaxVecCols : MPCG_MAX_COLS;
  if (B < 1 || B > maxb || opts->epochs < 0) {
    set_err("batch must be in 1..%d and epochs >= 0", maxb);
    return MPCG_ERR_ARG;
  }
  for (int i = 0; i < nprob; ++i) {
    CKS(check_h(hs[i]));
    CKS(net_check_grid(hs[i]));
    const GridDesc& gi = hs[i]->lev[hs[i]->levels - 1].g;
    const GridDesc& g0 = hs[0]->lev[hs[0]->levels - 1].g;
    if (net3_of(hs[i]) != net3 || gi.nx != g0.nx || gi.ny != g0.ny || gi.nz != g0.nz || gi.ncomp != g0.ncomp) {
      set_err("all training problems must share the fine grid");
      return MPCG_ERR_ARG;
    }
  }
  for (int i = 0; i < npairs; ++i)
    if (pair_prob[i] < 0 || pair_prob[i] >= nprob) {
      set_err("pair_prob[%d] out of range", i);
      return MPCG_ERR_ARG;
    }
  mg_hierarchy* h0 = hs[0];
  CK(cudaSetDevice(h0->device));
  cudaStream_t s = h0->stream;
  const GridDesc g = h0->lev[h0->levels - 1].g;
  if (!net3 && g.p > 1024) {
    set_err("training grids are limited to 1025 nodes per side");
    return MPCG_ERR_ARG;
  }
  for (int i = 0; i < nprob; ++i) {
    CKS(build_f32(hs[i]));
    CKS(net_prepare(hs[i]));
  }
  Alloc mem;
  NetBatch nbt;
  mpcg_status st = net_batch_alloc(net3, g, B, mem, s, nbt);
  auto get = [&](auto** p, size_t n) {
    if (st == MPCG_OK) st = mem.get(p, n, s);
  };
  float *R, *E, *AE, *master, *m, *v, *wq;
  double* loss;
  const size_t L = g.len;
  get(&R, (size_t)npairs * L);
  get(&E, (size_t)npairs * L);
  get(&AE, (size_t)npairs * L);
  get(&master, nbt.np);
  get(&m, nbt.np);
  get(&v, nbt.np);
  get(&wq, nbt.np);
  get(&loss, 1);
  if (st != MPCG_OK) {
    mem.release();
    return st;
  }
  copy_floats(master, params, nbt.np, s);
  launch_round_bf16(master, wq, nbt.np, s);
  // training set in the padded layout, and A e per pair (FP32 operators)
  launch_pack<float, float>(g, rhat_dev, g.n, R, npairs, s);
  launch_pack<float, float>(g, e_dev, g.n, E, npairs, s);
  for (int i = 0; i < npairs; ++i) {
    const Level& Lp = hs[pair_prob[i]]->lev[hs[pair_prob[i]]->levels - 1];
    launch_spmm<float>(g, Lp.st32, E + (size_t)i * L, AE + (size_t)i * L, 1, nullptr, nullptr, s);
  }
  // batches: pairs grouped by problem, shuffled within a problem and across
  // batches by a seeded 64-bit LCG (Knuth's MMIX constants)
  unsigned long long lcg = opts->seed * 2862933555777941757ULL + 3037000493ULL;
  auto rnd = [&](unsigned long long n) {
    lcg = lcg * 6364136223846793005ULL + 1442695040888963407ULL;
    return (lcg >> 33) % n;
  };
  std::vector<std::vector<int>> byprob(nprob);
  for (int i = 0; i < npairs; ++i) byprob[pair_prob[i]].push_back(i);
  int step = 0;
  for (int ep = 0; ep < opts->epochs && st == MPCG_OK; ++ep) {
    std::vector<std::vector<int>> batches;
    for (auto& lst : byprob) {
      for (size_t i = lst.size(); i > 1; --i) std::swap(lst[i - 1], lst[rnd(i)]);
      for (size_t i = 0; i < lst.size(); i += B)
        batches.emplace_back(lst.begin() + i, lst.begin() + std::min(lst.size(), i + (size_t)B));
    }
    for (size_t i = batches.size(); i > 1; --i) std::swap(batches[i - 1], batches[rnd(i)]);
    cudaMemsetAsync(loss, 0, sizeof(double), s);
    for (auto& bt : batches) {
      const int nb = (int)bt.size();
      for (int k = 0; k < nb; ++k) {
        cudaMemcpyAsync(nbt.rb + k * L, R + (size_t)bt[k] * L, sizeof(float) * L, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(nbt.eb + k * L, E + (size_t)bt[k] * L, sizeof(float) * L, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(nbt.aeb + k * L, AE + (size_t)bt[k] * L, sizeof(float) * L, cudaMemcpyDeviceToDevice, s);
      }
      mg_hierarchy* hp = hs[pair_prob[bt[0]]];
      net_batch_step(nbt, g, nb, hp->net_c, hp->lev[hp->levels - 1].st32, wq, loss, s);
      ++step;
      // a short last batch of a problem launches fewer blocks
      launch_net_adam(nbt.parts_dev, net_batch_blocks(nbt, g, nb), net3 ? 1 : 0, master, m, v, wq, step,
                      (float)opts->lr, (float)opts->beta1, (float)opts->beta2, (float)opts->eps, s);
    }
    double lh = 0.0;
    int terr_h = 0;
    if (cudaMemcpyAsync(&lh, loss, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&terr_h, nbt.terr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      set_err("training step failed: %s", cudaGetErrorString(cudaGetLastError()));
      st = MPCG_ERR_CUDA;
      break;
    }
    if (terr_h) {
      set_err("training: a tensor-core wait timed out");
      st = MPCG_ERR_TIMEOUT;
      break;
    }
    if (loss_hist) loss_hist[ep] = lh / (double)batches.size();
  }
  if (st == MPCG_OK) {
    cudaMemcpyAsync(params, master, sizeof(float) * nbt.np,
                    is_device_pointer(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) st = MPCG_ERR_CUDA;
  }
  mem.release();
  return st;
}

}  // extern "C"

namespace mpcg {
bool batched_graph_eligible(mg_hierarchy* const* hs, int nclass) { return classes_graph_eligible(hs, nclass); }
}  // namespace mpcg
