// C ABI of libslm (include/slm.h): argument checks, staging of host arrays,
// the batched swarm search driver, and level-by-level tree growth.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <numeric>
#include <random>
#include <string>
#include <type_traits>
#include <vector>

#include "slm_internal.cuh"

using namespace slm;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

// A level's search folds the move into the projection when its projection
// is at most this many waves of row-tile units (slm_set_fused_step, on = 1).
constexpr int kFusedMaxWaves = 4;
// The fixed cost of one folded projection unit, in rows of work.
constexpr int kStepUnitRows = 32;

enum Slot {
  W_X, W_LAB, W_Y, W_IDX, W_W, W_BINS, W_XL, W_LABL, W_YL,
  S_POS, S_VEL, S_PBEST, S_GBEST, S_CUR, S_PB, S_GB, S_GPART, S_GITER,
  S_TRACE, S_ZMM, S_Z, S_DONE, S_NODES, S_TILES, S_STATUS, S_ERR, S_OUT,
  // SLM_PROJ_BF16_TOPK
  W_XB, S_POSB, S_MTILES, S_SEL, S_INV, S_POSK, S_Z2, S_ZMM2, S_CUR2,
  // MSE moments
  S_M1, S_M2, S_MACCW, S_MACCY, S_MSCALE,
  // learned proposal: node statistics, network work space, training data
  S_PSTATS, S_PYR, S_PACC, S_PWK, S_PWORK, S_PLOSS, W_PS, W_PD, W_PT, W_PIDX, W_PBS, W_PBD,
  W_PBT, W_PRHO, W_PMU, W_PPOS,
  // node lists of the histogram kernels (large nodes, then small ones) and
  // of the persistent search
  S_HLIST, S_NLIST,
  // feature pre-screen: unit positions, kept features, the kept columns,
  // the lifted gbest
  S_FPOS, S_FEAT, W_XS, S_GFULL,
  // adaptive PSO state per node
  S_APSO,
  // the projection with the move folded in: second position buffer, the
  // gB-independent move terms, its row tiles
  S_POS2, S_IC, S_S2, S_STILES, S_IMP,
  // probabilistic search: every candidate's vector and score, the rank
  // tables, the best so far, the pruning's state
  S_PRALL, S_PRSC, S_PRTAB, S_PRBEST, S_PRUNE,
  // a level's growth (slm_grow_level): node list, statistics, split flags,
  // per-tile accumulators, the partition's lists (reused by every forest)
  S_GLVLNODES, S_GLVLSPLIT, S_GLVLCLS, S_GLVLPAR, S_GSMAP, S_GOUT3, S_GDST, S_GLTILES, S_GLTILE0,
  S_GACCW, S_GACCY, S_GTILESUM, S_GSTILE0, S_GTILELEFT, S_GTILEBASE, S_GPLK, S_GPWL,
  N_SLOTS
};

}  // namespace

struct slm_ctx {
  int device = 0;
  int n_sm = 1;
  cudaStream_t stream = nullptr;
  std::string err;
  DevBuf ws[N_SLOTS];
  // launch accounting and optional per-kernel CUDA-event timing
  int64_t launches = 0;
  bool prof = false;
  struct Pending {
    int kid;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;
  int64_t k_launches[SLM_K_COUNT] = {};
  double k_ms[SLM_K_COUNT] = {};
  double k_pairs[SLM_K_COUNT] = {};
  const slm_proposal* prop = nullptr;  // seeds searches with params.seeded
  // projection tiles: picked per problem shape by timing the candidates on
  // the first search of that shape (tune = 1), or fixed (tune = 0)
  struct Tiles {
    int pg = kPG;        // particles per group
    int cps = 2;         // CTAs per SM of the persistent grid
    float ms = 0.f;      // tuned: time of two projections with these tiles
    bool gather = false; // rows gathered from the base rows by sample id
    bool tma = true;     // contiguous rows staged by tensor-map tile copies
  };
  int tune = 1;
  // histogram clusters: CTAs per (node, particle), tuned per shape
  struct Split {
    int S = 1;
    float ms = 0.f;
  };
  std::map<std::vector<int64_t>, Split> tuned_split;
  int last_split = 0;
  bool node_search = false;           // persistent search of the nodes that fit
  int last_node_search = 0;           // CTAs per node of the last search (0: none)
  cudaStream_t side = nullptr;        // the persistent search beside the others
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int small_node_max = kWarpNodeMax;  // warp-per-particle histograms up to this,
  int64_t small_min_pairs = -1;       // for at least this many (node, particle)
                                      // pairs (-1: 2 x SMs x warps per CTA)
  Tiles forced{0, 0};
  std::map<uint64_t, Tiles> tuned;
  Tiles cur{};   // tiles of the search in flight
  Tiles last{};  // tiles of the last search
  // a search's iteration loop as one CUDA graph launch (reused executable)
  bool graphs = false;
  // FP32 projection of contiguous rows staged by tensor-map tile copies
  bool tma = true;
  // plain FP32 searches with the swarm move folded into the projection
  // (k_step: two launches per iteration instead of three)
  int fused_step = 1;  // 0 off, 1 when the level's projection is short, 2 always
  int step_shape = -1;      // k_step tile shape forced (-1: chosen per batch)
  int last_step_shape = -1;
  int64_t fused_searches = 0;
  // classification searches score with k_hist_cls (else k_hist_scan)
  bool class_hist = true;
  // folded searches whose nodes all take k_hist_cls: the move in its last
  // CTA per node (else in every k_step CTA)
  bool node_step = false;
  // global tree id of a forest's local tree t: tree_id0 + t * tree_stride
  // (a forest split across processes grows trees r, r + N, ... on rank r)
  int64_t tree_id0 = 0, tree_stride = 1;
  cudaStream_t cap_stream = nullptr;  // records graphs (the caller's stream may
                                      // be the legacy default stream)
  // executable graphs by launch signature (every kernel node's function,
  // grid, block, shared memory and cluster shape, in order): a new capture
  // with a known signature differs only in kernel arguments and updates that
  // executable in place
  struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::string key;            // launch inputs it was last recorded from
    std::vector<uint64_t> sig;  // launch signature
    int64_t launches = 0;       // kernel launches per graph launch
    int64_t k_launches[SLM_K_COUNT] = {};
    double k_pairs[SLM_K_COUNT] = {};
  };
  std::vector<GraphEntry> graph_cache;
  int64_t graph_launches = 0, graph_reuses = 0, graph_updates = 0, graph_instantiations = 0;
};

// Learned swarm proposal: FP32 parameters, their bfloat16 copies, gradients
// and Adam moments in one device allocation.
struct slm_proposal {
  int device = 0;
  DevBuf mem;
  MlpParams m{};
  MlpGrads g{};
  MlpState s{};
  int64_t step = 0;  // Adam steps taken
};

struct slm_forest {
  slm_ctx* ctx = nullptr;  // creating context (not owned; may be gone at free)
  int device = 0;
  slm_params params{};
  int64_t n = 0;
  int d = 0;
  int H = 0;
  int n_trees = 0;
  int K = 0;
  // the base rows, kept by bagged forests whose rows fit in a quarter of L2:
  // a level's FP32 projection may gather them by sample id instead of
  // reading the level's entry-ordered copy (which holds each tree's rows)
  const float* X = nullptr;
  DevBuf own_X;
  TreeArrays tr{};
  DevBuf tree_mem;
  // level-resident entry arrays, ping-pong
  DevBuf lX[2], lab[2], ly[2], lw[2], lidx[2], side;
  DevBuf lXb;     // bfloat16 rows of the current level (SLM_PROJ_BF16_TOPK)
  int align = 4;  // node segments start on multiples of this many entries
  int64_t tree_id0 = 0, tree_stride = 1;  // global id of local tree t
  uint32_t tree_id(int t) const { return (uint32_t)(tree_id0 + (int64_t)t * tree_stride); }
  int cur = 0;
  bool weighted = false;
  std::vector<LevelNode> level;  // nodes of the level to grow next
  int depth = 0;
  bool done = false;
  int64_t evaluations = 0;
  std::vector<int64_t> tree_evals;  // evaluations per tree
};

namespace {

static_assert(sizeof(slm_params) == 80 && offsetof(slm_params, apso) == 64 &&
                  offsetof(slm_params, seed) == 72,
              "slm_params layout is part of the ABI (bindings mirror it)");

slm_status fail(slm_ctx* c, slm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

slm_status cuda_fail(slm_ctx* c, cudaError_t e, const char* where) {
  if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SLM_ENOMEM : SLM_ECUDA;
}

#define CK(expr)                                    \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #expr); \
  } while (0)

// Test hook: the next `g_fail_alloc`-th growth of a work buffer fails as if
// the device were out of memory (0: never).
std::atomic<int64_t> g_fail_alloc{0};

cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (bytes <= b.cap) return cudaSuccess;
  if (g_fail_alloc.load() > 0 && g_fail_alloc.fetch_sub(1) == 1) return cudaErrorMemoryAllocation;
  if (b.p) {
    cudaError_t e = cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    if (e) return e;
  }
  const size_t want = bytes + bytes / 4;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e) {
    b.p = nullptr;
    return e;
  }
  b.cap = want;
  return cudaSuccess;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller array: the pointer itself, or a staged copy.
template <typename T>
slm_status stage_in(slm_ctx* c, const T* src, size_t count, DevBuf& buf,
                    const T** out) {
  if (!src || count == 0) {
    *out = src;
    return SLM_OK;
  }
  if (is_device_ptr(src)) {
    *out = src;
    return SLM_OK;
  }
  CK(ensure(buf, sizeof(T) * count));
  CK(cudaMemcpyAsync(buf.p, src, sizeof(T) * count, cudaMemcpyHostToDevice,
                     c->stream));
  *out = static_cast<const T*>(buf.p);
  return SLM_OK;
}

int round16(int v) { return (v + 15) / 16 * 16; }

// The tensor-core pass stages all positions of a node in shared memory.
slm_status check_bf16_size(slm_ctx* c, int d, int P) {
  if ((int64_t)round16(P) * round16(d) * 2 > kMmaMaxBBytes)
    return fail(c, SLM_EUNSUPPORTED,
                "SLM_PROJ_BF16_TOPK needs round16(n_particles) * round16(d) * 2 <= 131072");
  return SLM_OK;
}

slm_status check_params(slm_ctx* c, const slm_params* p, int32_t d,
                        bool need_swarm) {
  if (!p) return fail(c, SLM_EINVAL, "params is NULL");
  if (p->criterion < SLM_GINI || p->criterion > SLM_MSE)
    return fail(c, SLM_EINVAL, "criterion out of range");
  if (p->criterion != SLM_MSE && (p->n_classes < 2 || p->n_classes > kMaxClasses))
    return fail(c, SLM_EINVAL, "n_classes must be in [2, 32]");
  if (p->n_bins < 2 || p->n_bins > kMaxBins)
    return fail(c, SLM_EINVAL, "n_bins must be in [2, 256]");
  if (p->criterion != SLM_MSE &&
      (int64_t)p->n_bins * p->n_classes * 4 > kMaxHistBytesPerParticle)
    return fail(c, SLM_EUNSUPPORTED, "n_bins * n_classes * 4 exceeds 10240");
  if (p->min_leaf < 1) return fail(c, SLM_EINVAL, "min_leaf must be >= 1");
  if (d < 1 || d > kMaxD) return fail(c, SLM_EINVAL, "d must be in [1, 1024]");
  if (need_swarm) {
    if (p->n_particles < 1 || p->n_particles > kMaxParticles)
      return fail(c, SLM_EINVAL, "n_particles must be in [1, 256]");
    if (p->n_iters < 0) return fail(c, SLM_EINVAL, "n_iters must be >= 0");
    if (p->proj != SLM_PROJ_FP32 && p->proj != SLM_PROJ_BF16_TOPK)
      return fail(c, SLM_EINVAL, "proj must be SLM_PROJ_FP32 or SLM_PROJ_BF16_TOPK");
    if (p->proj == SLM_PROJ_BF16_TOPK) {
      if (p->topk < 1 || p->topk > p->n_particles)
        return fail(c, SLM_EINVAL, "topk must be in [1, n_particles]");
      if (slm_status s = check_bf16_size(c, d, p->n_particles)) return s;
    }
    if (!std::isfinite(p->inertia) || !std::isfinite(p->c1) ||
        !std::isfinite(p->c2))
      return fail(c, SLM_EINVAL, "inertia / c1 / c2 must be finite");
    if (p->seeded != 0 && p->seeded != 1) return fail(c, SLM_EINVAL, "seeded must be 0 or 1");
    if (p->top_n < 0) return fail(c, SLM_EINVAL, "top_n must be >= 0");
    if (p->apso != 0 && p->apso != 1) return fail(c, SLM_EINVAL, "apso must be 0 or 1");
    if (p->apso && (p->proj != SLM_PROJ_FP32 || p->n_particles >= kMaxParticles ||
                    (size_t)((p->n_particles + 3) & ~3) * d * 4 > 200 * 1024))
      return fail(c, SLM_EUNSUPPORTED,
                  "adaptive PSO needs SLM_PROJ_FP32, n_particles < 256 and (n_particles "
                  "rounded up to 4) * d * 4 <= 200 KB");
    if (p->top_n > 0 && p->top_n < d &&
        (p->proj != SLM_PROJ_FP32 || p->seeded || d > kMaxParticles))
      return fail(c, SLM_EUNSUPPORTED,
                  "a feature pre-screen (0 < top_n < d) needs SLM_PROJ_FP32, seeded = 0, "
                  "d <= 256");
    if (p->seeded) {
      if (!c->prop) return fail(c, SLM_EINVAL, "seeded search without slm_use_proposal");
      if (d > kPropD || (p->criterion != SLM_MSE && p->n_classes > kPropK) ||
          p->n_particles > kPropP)
        return fail(c, SLM_EUNSUPPORTED,
                    "seeded searches need d <= 256, n_classes <= 20, n_particles <= 64");
    }
  }
  return SLM_OK;
}

cudaEvent_t take_event(slm_ctx* c) {
  if (!c->free_events.empty()) {
    cudaEvent_t e = c->free_events.back();
    c->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Runs one kernel launch, counting it and (when profiling) bracketing it with
// events on the context's stream. pairs: particle-sample pairs it scores.
template <class F>
cudaError_t launch(slm_ctx* c, int kid, double pairs, F&& fn) {
  c->launches += 1;
  c->k_launches[kid] += 1;
  c->k_pairs[kid] += pairs;
  if (!c->prof) return fn();
  cudaEvent_t ea = take_event(c), eb = take_event(c);
  if (ea) cudaEventRecord(ea, c->stream);
  cudaError_t e = fn();
  if (eb) cudaEventRecord(eb, c->stream);
  if (ea && eb) c->pending.push_back({kid, ea, eb});
  return e;
}

cudaError_t collect_profile(slm_ctx* c) {
  if (c->pending.empty()) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) return e;
  for (auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) c->k_ms[p.kid] += ms;
    c->free_events.push_back(p.a);
    c->free_events.push_back(p.b);
  }
  c->pending.clear();
  return cudaSuccess;
}

Problem make_problem(const slm_params* p, const float* X, int d, const int32_t* lab,
                     const float* y, const uint32_t* w, int64_t E, int P) {
  Problem pr{};
  pr.X = X;
  pr.lab = lab;
  pr.y = y;
  pr.w = w;
  pr.E = E;
  pr.Ez = (E + 3) / 4 * 4;
  pr.d = d;
  pr.crit = p->criterion;
  pr.K = p->criterion == SLM_MSE ? 1 : p->n_classes;
  pr.B = p->n_bins;
  pr.min_leaf = p->min_leaf;
  pr.P = P;
  pr.Pp = (P + kPG - 1) / kPG * kPG;
  pr.G = pr.Pp / kPG;
  return pr;
}

int64_t round_up(int64_t v, int64_t al) { return (v + al - 1) / al * al; }

// Entries the level arrays need: the root's (padded) entries plus the
// padding of every node of a level (< align each), plus a 16-byte guard. A
// level holds at most n_trees 2^max_depth nodes, and (unweighted) every node
// below the root holds at least min_leaf entries.
int64_t level_capacity(int64_t e_root, int n_trees, int max_depth, int align, int min_leaf,
                       bool weighted) {
  int64_t nodes = (int64_t)n_trees << max_depth;
  const int64_t by_size = weighted ? e_root : n_trees + e_root / (min_leaf > 0 ? min_leaf : 1);
  if (align > 4 && by_size < nodes) nodes = by_size;
  return e_root + (int64_t)align * nodes + 16;
}

// Projection work tiles: every node's segment cut into kTS-row tiles.
std::vector<WorkTile> plan_tiles(const std::vector<NodeDesc>& nodes) {
  std::vector<WorkTile> t;
  for (int a = 0; a < (int)nodes.size(); ++a)
    for (int s = 0; s < nodes[a].seg_len; s += kTS)
      t.push_back(WorkTile{a, nodes[a].seg_start + s, std::min(kTS, nodes[a].seg_len - s), 0});
  return t;
}

template <typename T>
T* ws_ptr(slm_ctx* c, Slot s) {
  return static_cast<T*>(c->ws[s].p);
}

// Scoring buffers of A nodes (one batch): z, ranges, node and tile lists;
// for MSE also the entries' fixed-point moments (pr.m1, pr.m2, pr.mscale).
slm_status setup_scoring(slm_ctx* c, Problem& pr, int A,
                         const std::vector<NodeDesc>& nodes,
                         const std::vector<WorkTile>& tiles, Swarm* sw) {
  CK(ensure(c->ws[S_CUR], sizeof(EvalRes) * (size_t)A * pr.Pp));
  CK(ensure(c->ws[S_ZMM], sizeof(int32_t) * 2 * (size_t)A * pr.Pp));
  CK(ensure(c->ws[S_Z], sizeof(float) * (size_t)pr.P * (size_t)(pr.Ez > 0 ? pr.Ez : 4)));
  CK(ensure(c->ws[S_NODES], sizeof(NodeDesc) * nodes.size()));
  CK(ensure(c->ws[S_TILES], sizeof(WorkTile) * tiles.size()));
  CK(cudaMemcpyAsync(c->ws[S_NODES].p, nodes.data(), sizeof(NodeDesc) * nodes.size(),
                     cudaMemcpyHostToDevice, c->stream));
  if (!tiles.empty())
    CK(cudaMemcpyAsync(c->ws[S_TILES].p, tiles.data(), sizeof(WorkTile) * tiles.size(),
                       cudaMemcpyHostToDevice, c->stream));
  CK(ensure(c->ws[S_ERR], sizeof(int32_t)));
  CK(cudaMemsetAsync(c->ws[S_ERR].p, 0, sizeof(int32_t), c->stream));
  if (pr.crit == SLM_MSE) {
    const size_t ne = (size_t)(pr.Ez > 0 ? pr.Ez : 4) + 16;
    CK(ensure(c->ws[S_M1], sizeof(long long) * ne));
    CK(ensure(c->ws[S_M2], sizeof(long long) * ne));
    CK(ensure(c->ws[S_MACCW], sizeof(unsigned long long) * (size_t)A));
    CK(ensure(c->ws[S_MACCY], sizeof(int32_t) * 2 * (size_t)A));
    CK(ensure(c->ws[S_MSCALE], sizeof(double) * 2 * (size_t)A));
    pr.m1 = ws_ptr<long long>(c, S_M1);
    pr.m2 = ws_ptr<long long>(c, S_M2);
    pr.mscale = ws_ptr<double>(c, S_MSCALE);
    CK(launch(c, SLM_K_NODE_STATS, 0.0, [&] {
      return launch_mse_moments(pr, ws_ptr<WorkTile>(c, S_TILES), (int)tiles.size(), A,
                                ws_ptr<unsigned long long>(c, S_MACCW),
                                ws_ptr<int32_t>(c, S_MACCY), ws_ptr<long long>(c, S_M1),
                                ws_ptr<long long>(c, S_M2), ws_ptr<double>(c, S_MSCALE),
                                c->stream);
    }));
  }
  sw->cur = ws_ptr<EvalRes>(c, S_CUR);
  sw->zmm = ws_ptr<int32_t>(c, S_ZMM);
  sw->z = ws_ptr<float>(c, S_Z);
  sw->err = ws_ptr<int32_t>(c, S_ERR);
  CK(prepare_eval_kernels(pr));
  return SLM_OK;
}

// Allocates the swarm buffers of A nodes.
slm_status setup_swarm(slm_ctx* c, Problem& pr, int A, int T, bool want_trace,
                       const std::vector<NodeDesc>& nodes,
                       const std::vector<WorkTile>& tiles, Swarm* sw) {
  Swarm s{};
  if (slm_status st = setup_scoring(c, pr, A, nodes, tiles, &s)) return st;
  const size_t apd = (size_t)A * pr.Pp * pr.d;
  CK(ensure(c->ws[S_POS], sizeof(float) * apd));
  CK(ensure(c->ws[S_VEL], sizeof(float) * apd));
  CK(ensure(c->ws[S_PBEST], sizeof(float) * apd));
  CK(ensure(c->ws[S_GBEST], sizeof(float) * (size_t)A * pr.d));
  CK(ensure(c->ws[S_PB], sizeof(EvalRes) * (size_t)A * pr.Pp));
  CK(ensure(c->ws[S_GB], sizeof(EvalRes) * 2 * (size_t)A));
  CK(ensure(c->ws[S_GPART], sizeof(int32_t) * (size_t)A));
  CK(ensure(c->ws[S_GITER], sizeof(int32_t) * (size_t)A));
  CK(ensure(c->ws[S_DONE], sizeof(int32_t) * (size_t)A));
  CK(cudaMemsetAsync(c->ws[S_DONE].p, 0, sizeof(int32_t) * (size_t)A, c->stream));
  if (want_trace) CK(ensure(c->ws[S_TRACE], sizeof(double) * (size_t)A * (T + 1)));
  CK(ensure(c->ws[S_APSO], sizeof(ApsoState) * (size_t)A));
  s.pos = ws_ptr<float>(c, S_POS);
  s.vel = ws_ptr<float>(c, S_VEL);
  s.pbest = ws_ptr<float>(c, S_PBEST);
  s.gbest = ws_ptr<float>(c, S_GBEST);
  s.pb = ws_ptr<EvalRes>(c, S_PB);
  s.gb = ws_ptr<EvalRes>(c, S_GB);
  s.gpart = ws_ptr<int32_t>(c, S_GPART);
  s.giter = ws_ptr<int32_t>(c, S_GITER);
  s.done = ws_ptr<int32_t>(c, S_DONE);
  s.trace = want_trace ? ws_ptr<double>(c, S_TRACE) : nullptr;
  s.T = T;
  *sw = s;
  return SLM_OK;
}

// Cluster split of the histogram kernel for a batch.
int batch_split(slm_ctx* c, const Problem& pr, const std::vector<NodeDesc>& nodes) {
  int64_t max_len = 0;
  for (const NodeDesc& nd : nodes) max_len = std::max<int64_t>(max_len, nd.seg_len);
  return hist_split(pr, (int)nodes.size(), max_len, c->n_sm, hist_max_cluster(pr));
}

// The reduced-precision pass of SLM_PROJ_BF16_TOPK: bfloat16 scores of all
// particles on the tensor cores, then FP32 re-scores of the k best per node.
struct Bf16Plan {
  bool on = false;
  int k = 0, kp = 0;     // re-scored particles per node; padded to 8
  int n_mtiles = 0;      // kMmaRows-row tiles of the batch
  int grid = 0;          // k_project_mma grid
  int S_k = 1;           // cluster split of the re-scoring histogram pass
  double pairs_k = 0.0;
  Problem pr_k{};        // the re-scoring problem: P = k
  Swarm sw_k{};          // its view: compact positions, z, ranges, scores
  uint16_t* posb = nullptr;
  int32_t* sel = nullptr;
  int32_t* inv = nullptr;
  // both passes on the histogram kernels of k_hist_cls (squared error or
  // class counts; the reduced pass's last CTA per node selecting the top
  // k), splits S_fast / S_fast_k, the c ln c table of entropy scans
  bool fast = false;
  int S_fast = 1, S_fast_k = 1;
  const double* xtab = nullptr;
};

// Histogram kernels of a classification search: the nodes of at most
// small_node_max entries go to the warp-per-particle kernel, the others to
// the cluster kernel.
struct HistPlan {
  bool on = false;
  const int32_t* large = nullptr;  // cluster kernel
  int n_large = 0, S_large = 1;
  double pairs_large = 0.0;
  const int32_t* small = nullptr;  // warp kernel
  int n_small = 0;
  double pairs_small = 0.0;
  const int32_t* moved = nullptr;  // the swarm update's nodes (null: all)
  int n_moved = 0;
  int64_t max_large = 0;           // largest node of the cluster kernel's list
};

// Classification histograms by k_hist_cls: its cluster sizes for all nodes
// of the batch and for a HistPlan's large list.
struct ClsPlan {
  bool on = false;
  int S = 1, S_large = 1;
  const double* xtab = nullptr;
};

// Lists of the histogram kernels and the swarm update for the nodes `in`
// marks (all when empty): set when only some nodes of the batch run the
// per-iteration kernels, or when enough small nodes take the warp kernel.
slm_status setup_hist_plan(slm_ctx* c, const Problem& pr, const std::vector<NodeDesc>& nodes,
                           const std::vector<char>& in, HistPlan* plan) {
  *plan = HistPlan{};
  const bool subset = !in.empty();
  auto member = [&](int a) { return !subset || in[a] != 0; };
  const bool warp_ok = c->small_node_max > 0 && hist_warp_ok(pr);
  std::vector<int32_t> large, small;
  int64_t max_large = 0;
  for (int a = 0; a < (int)nodes.size(); ++a) {
    if (!member(a)) continue;
    if (warp_ok && nodes[a].seg_len <= c->small_node_max) {
      small.push_back(a);
      plan->pairs_small += (double)nodes[a].seg_len * pr.P;
    } else {
      large.push_back(a);
      max_large = std::max<int64_t>(max_large, nodes[a].seg_len);
      plan->pairs_large += (double)nodes[a].seg_len * pr.P;
    }
  }
  const int64_t min_pairs =
      c->small_min_pairs >= 0 ? c->small_min_pairs : 2LL * c->n_sm * (kThreads / 32);
  if ((int64_t)small.size() * pr.P < min_pairs) {  // too few for the warp kernel
    for (int32_t a : small) {
      large.push_back(a);
      max_large = std::max<int64_t>(max_large, nodes[a].seg_len);
    }
    plan->pairs_large += plan->pairs_small;
    plan->pairs_small = 0.0;
    small.clear();
    std::sort(large.begin(), large.end());
  }
  if (!subset && small.empty()) return SLM_OK;  // the cluster kernel on every node
  std::vector<int32_t> lst(large);
  lst.insert(lst.end(), small.begin(), small.end());
  std::vector<int32_t> moved;
  for (int a = 0; a < (int)nodes.size(); ++a)
    if (member(a)) moved.push_back(a);
  lst.insert(lst.end(), moved.begin(), moved.end());
  CK(ensure(c->ws[S_HLIST], sizeof(int32_t) * lst.size()));
  CK(cudaMemcpyAsync(c->ws[S_HLIST].p, lst.data(), sizeof(int32_t) * lst.size(),
                     cudaMemcpyHostToDevice, c->stream));
  const int32_t* base = static_cast<const int32_t*>(c->ws[S_HLIST].p);
  plan->large = base;
  plan->n_large = (int)large.size();
  plan->max_large = max_large;
  plan->small = base + large.size();
  plan->n_small = (int)small.size();
  if (subset) {
    plan->moved = base + large.size() + small.size();
    plan->n_moved = (int)moved.size();
  }
  if (plan->n_large)
    plan->S_large = hist_split(pr, plan->n_large, max_large, c->n_sm, hist_max_cluster(pr));
  plan->on = true;
  return SLM_OK;
}

// Buffers of the reduced-precision pass for A nodes whose segments start on
// multiples of kMmaRows; sw->sel / sw->k are set for a search.
slm_status setup_bf16(slm_ctx* c, const Problem& pr, const std::vector<NodeDesc>& nodes,
                      int k, bool search, Swarm* sw, Bf16Plan* plan) {
  const int A = (int)nodes.size();
  Bf16Plan b;
  b.on = true;
  b.k = k;
  b.kp = (k + 7) / 8 * 8;  // the re-scoring projection runs in groups of 8 or 16
  std::vector<WorkTile> mt;
  for (int a = 0; a < A; ++a) {
    if (nodes[a].seg_start % kMmaRows)
      return fail(c, SLM_ECUDA, "internal: node segment not aligned for the tensor-core pass");
    for (int r = 0; r < nodes[a].seg_len; r += kMmaRows)
      mt.push_back(WorkTile{a, nodes[a].seg_start + r, std::min(kMmaRows, nodes[a].seg_len - r), 0});
    b.pairs_k += (double)nodes[a].seg_len * k;
  }
  b.n_mtiles = (int)mt.size();
  CK(ensure(c->ws[S_MTILES], sizeof(WorkTile) * mt.size()));
  if (!mt.empty())
    CK(cudaMemcpyAsync(c->ws[S_MTILES].p, mt.data(), sizeof(WorkTile) * mt.size(),
                       cudaMemcpyHostToDevice, c->stream));
  CK(ensure(c->ws[S_POSB], sizeof(uint16_t) * (size_t)A * pr.Pp * pr.dp));
  b.posb = ws_ptr<uint16_t>(c, S_POSB);
  CK(prepare_mma_kernels(pr));
  const int cap = mma_grid_cap(pr, c->n_sm);
  if (cap < 1) return fail(c, SLM_EUNSUPPORTED, "the tensor-core pass cannot be scheduled");
  b.grid = std::min(cap, std::max(1, b.n_mtiles));
  if (k > 0) {
    CK(ensure(c->ws[S_SEL], sizeof(int32_t) * (size_t)A * k));
    CK(ensure(c->ws[S_INV], sizeof(int32_t) * (size_t)A * pr.Pp));
    CK(ensure(c->ws[S_POSK], sizeof(float) * (size_t)A * b.kp * pr.d));
    CK(ensure(c->ws[S_Z2], sizeof(float) * (size_t)k * (size_t)(pr.Ez > 0 ? pr.Ez : 4)));
    CK(ensure(c->ws[S_ZMM2], sizeof(int32_t) * 2 * (size_t)A * b.kp));
    CK(ensure(c->ws[S_CUR2], sizeof(EvalRes) * (size_t)A * b.kp));
    std::vector<int32_t> zinit(2 * (size_t)A * b.kp);
    for (size_t i = 0; i < zinit.size(); i += 2) {
      zinit[i] = INT32_MAX;
      zinit[i + 1] = INT32_MIN;
    }
    CK(cudaMemcpyAsync(c->ws[S_ZMM2].p, zinit.data(), sizeof(int32_t) * zinit.size(),
                       cudaMemcpyHostToDevice, c->stream));
    CK(ensure(c->ws[S_DONE], sizeof(int32_t) * (size_t)A));
    CK(cudaMemsetAsync(c->ws[S_DONE].p, 0, sizeof(int32_t) * (size_t)A, c->stream));
    b.sel = ws_ptr<int32_t>(c, S_SEL);
    b.inv = ws_ptr<int32_t>(c, S_INV);
    b.pr_k = pr;
    b.pr_k.P = k;
    b.pr_k.Pp = b.kp;
    b.pr_k.G = b.kp % 16 == 0 ? b.kp / 16 : b.kp / 8;
    // the re-scoring pass: compact positions, its own z, ranges and scores
    b.sw_k = *sw;
    b.sw_k.pos = ws_ptr<float>(c, S_POSK);
    b.sw_k.z = ws_ptr<float>(c, S_Z2);
    b.sw_k.zmm = ws_ptr<int32_t>(c, S_ZMM2);
    b.sw_k.cur = ws_ptr<EvalRes>(c, S_CUR2);
    b.sw_k.sel = nullptr;
    b.sw_k.tk_sel = nullptr;
    b.sw_k.posb = nullptr;
    b.S_k = batch_split(c, b.pr_k, nodes);
    // the reduced pass's histogram kernel selects each node's top k
    sw->done = ws_ptr<int32_t>(c, S_DONE);
    sw->tk_sel = b.sel;
    sw->tk_inv = b.inv;
    sw->tk_pos = ws_ptr<float>(c, S_POSK);
    sw->tk_k = k;
    sw->tk_kp = b.kp;
    if (search) {
      sw->sel = b.sel;
      sw->k = k;
    }
  }
  if (search) sw->posb = b.posb;  // written by the swarm kernels
  *plan = b;
  return SLM_OK;
}

// A plain FP32 search whose move is folded into the projection (k_step):
// positions alternate between pos[0] and pos[1] by iteration parity.
struct StepPlan {
  bool on = false;
  float* pos[2] = {nullptr, nullptr};
  const WorkTile* tiles = nullptr;
  int n_tiles = 0;
  int grid = 0;
  int sh = 0;  // tile shape of k_step
};

// One scoring pass of every (node, particle) of a batch; with a swarm
// (co != null) the pass ends with the swarm update of iteration t.
slm_status score_batch(slm_ctx* c, const Problem& pr, const Swarm& sw_in,
                       const std::vector<NodeDesc>& nodes, int n_tiles, double pairs,
                       int32_t* bins_out, int t, const SwarmCoef* co, int S,
                       const Bf16Plan* bp = nullptr, const HistPlan* hp = nullptr,
                       const StepPlan* sp = nullptr, const ClsPlan* cp = nullptr) {
  const int A = (int)nodes.size();
  const NodeDesc* dn = ws_ptr<NodeDesc>(c, S_NODES);
  const WorkTile* dt = ws_ptr<WorkTile>(c, S_TILES);
  const int cap = c->cur.cps * c->n_sm;
  Swarm sw = sw_in;
  if (sp && sp->on) {
    // iteration t: move (t > 0) and project in one launch; the histogram
    // kernels score x_t in pos[t & 1] and leave the next move's terms (or,
    // with node_step, move the swarm into pos[(t + 1) & 1] themselves)
    sw.pos = sp->pos[t & 1];
    sw.pos_next = sp->pos[(t + 1) & 1];
    const float* prev = sw.node_step ? sw.pos : sp->pos[t > 0 ? (t - 1) & 1 : 0];
    CK(launch(c, SLM_K_PROJECT, pairs, [&] {
      return launch_step(pr, sw, prev, dn, A, sp->tiles, sp->n_tiles, sp->grid, sp->sh, t,
                         c->stream);
    }));
  }
  if (bp && bp->on) {
    // bfloat16 scores of every particle on the tensor cores
    const Bf16Plan& b = *bp;
    if (!co)  // a search's positions are converted by its swarm kernels
      CK(launch(c, SLM_K_TOPK, 0.0, [&] {
        return launch_to_mma_layout(sw.pos, (int64_t)A * pr.Pp, pr.d, pr.dp, pr.Pp, A, b.posb,
                                    c->stream);
      }));
    if (b.n_mtiles)
      CK(launch(c, SLM_K_PROJECT_MMA, pairs, [&] {
        return launch_project_mma(pr, sw, ws_ptr<WorkTile>(c, S_MTILES), b.n_mtiles, b.posb,
                                  b.grid, c->stream);
      }));
    CK(launch(c, SLM_K_HIST_SCAN, pairs, [&] {
      return b.fast && !bins_out
                 ? launch_hist_cls(pr, sw, dn, A, b.S_fast, t, 0, b.xtab, c->stream)
                 : launch_hist_scan(pr, sw, dn, A, S, bins_out, t, 0, c->stream);
    }));
    if (b.k > 0) {
      // FP32 re-scores of the k best of each node (selected by the last
      // histogram CTA of the node) replace theirs
      if (n_tiles)
        CK(launch(c, SLM_K_PROJECT, b.pairs_k, [&] {
          return launch_project(b.pr_k, b.sw_k, dt, n_tiles, cap, c->stream, 0, false,
                                c->tma ? A : 0);
        }));
      CK(launch(c, SLM_K_HIST_SCAN, b.pairs_k, [&] {
        return b.fast
                   ? launch_hist_cls(b.pr_k, b.sw_k, dn, A, b.S_fast_k, t, 0, b.xtab, c->stream)
                   : launch_hist_scan(b.pr_k, b.sw_k, dn, A, b.S_k, nullptr, t, 0, c->stream);
      }));
      CK(launch(c, SLM_K_TOPK, 0.0, [&] {
        return launch_merge(pr, sw, A, b.sw_k.cur, b.kp, b.inv, t, co ? 1 : 0, c->stream);
      }));
    }
    if (co)
      CK(launch(c, SLM_K_SWARM_UPDATE, 0.0,
                [&] { return launch_move(pr, sw, dn, A, t, *co, c->stream); }));
    return SLM_OK;
  }
  if (n_tiles && !(sp && sp->on))
    CK(launch(c, SLM_K_PROJECT, pairs, [&] {
      return launch_project(pr, sw, dt, n_tiles, cap, c->stream, c->cur.pg, c->cur.gather,
                            c->tma && c->cur.tma ? A : 0);
    }));
  const bool cls = cp && cp->on && !bins_out;
  if (hp && hp->on && !bins_out) {
    if (hp->n_large)
      CK(launch(c, SLM_K_HIST_SCAN, hp->pairs_large, [&] {
        return cls ? launch_hist_cls(pr, sw, dn, hp->n_large, cp->S_large, t, co ? 1 : 0,
                                     cp->xtab, c->stream, hp->large)
                   : launch_hist_scan(pr, sw, dn, hp->n_large, hp->S_large, nullptr, t,
                                      co ? 1 : 0, c->stream, hp->large);
      }));
    if (hp->n_small)
      CK(launch(c, SLM_K_HIST_SCAN, hp->pairs_small, [&] {
        return launch_hist_warp(pr, sw, dn, hp->small, hp->n_small, t, co ? 1 : 0, c->stream);
      }));
  } else {
    CK(launch(c, SLM_K_HIST_SCAN, pairs, [&] {
      return cls ? launch_hist_cls(pr, sw, dn, A, cp->S, t, co ? 1 : 0, cp->xtab, c->stream)
                 : launch_hist_scan(pr, sw, dn, A, S, bins_out, t, co ? 1 : 0, c->stream);
    }));
  }
  // with adaptive PSO the evaluation scored the swarm's particles and the
  // elite slot after them; the swarm kernels see the particles only
  Problem psw = pr;
  if (sw.apso) psw.P = pr.P - 1;
  if (co && sw.apso)
    CK(launch(c, SLM_K_SWARM_UPDATE, 0.0, [&] {
      return launch_apso(psw, sw, dn, A, t, *co, c->stream, hp ? hp->moved : nullptr,
                         hp ? hp->n_moved : 0);
    }));
  // k_apso moves the adaptive swarm itself; a folded move needs only the
  // gbest step of the last evaluation
  if (co && !sw.apso && (!(sp && sp->on) || (t == sw.T && !sw.node_step)))
    CK(launch(c, SLM_K_SWARM_UPDATE, 0.0, [&] {
      return launch_move(psw, sw, dn, A, t, *co, c->stream, hp ? hp->moved : nullptr,
                         hp ? hp->n_moved : 0);
    }));
  return SLM_OK;
}

// Network work space for a batch of N samples.
slm_status proposal_work(slm_ctx* c, int N, MlpWork* w) {
  const size_t nh = (size_t)N * kPropH, no = (size_t)N * kPropOut;
  CK(ensure(c->ws[S_PWORK], sizeof(float) * (4 * nh + 2 * no)));
  float* b = ws_ptr<float>(c, S_PWORK);
  *w = MlpWork{b, b + nh, b + 2 * nh, b + 2 * nh + no, b + 2 * nh + 2 * no,
               b + 3 * nh + 2 * no};
  return SLM_OK;
}

// Statistics of the batch's nodes (already uploaded to S_NODES) into S_PSTATS.
slm_status batch_stats(slm_ctx* c, const Problem& pr, const std::vector<NodeDesc>& nodes,
                       float** stats) {
  const int A = (int)nodes.size();
  const int K = pr.lab ? pr.K : 4;
  int64_t max_len = 0;
  for (const NodeDesc& nd : nodes) max_len = std::max<int64_t>(max_len, nd.seg_len);
  CK(ensure(c->ws[S_PSTATS], sizeof(float) * (size_t)A * kPropIn));
  CK(ensure(c->ws[S_PYR], sizeof(int32_t) * 2 * (size_t)A));
  CK(ensure(c->ws[S_PACC], sizeof(double) * (size_t)A * (K + 2) * pr.d));
  CK(ensure(c->ws[S_PWK], sizeof(double) * (size_t)A * K));
  CK(launch(c, SLM_K_PROPOSAL, 0.0, [&] {
    return launch_node_stats(pr, ws_ptr<NodeDesc>(c, S_NODES), A, max_len, K,
                             ws_ptr<int32_t>(c, S_PYR), ws_ptr<double>(c, S_PACC),
                             ws_ptr<double>(c, S_PWK), ws_ptr<float>(c, S_PSTATS), c->n_sm,
                             c->stream);
  }));
  *stats = ws_ptr<float>(c, S_PSTATS);
  return SLM_OK;
}

// Initial swarms from the context's proposal: node statistics, the network,
// then positions around its direction (Sec. III-A's start, learned).
slm_status seed_swarms(slm_ctx* c, const Problem& pr, const std::vector<NodeDesc>& nodes,
                       const Swarm& sw, SwarmCoef co) {
  const int A = (int)nodes.size();
  float* stats = nullptr;
  if (slm_status s = batch_stats(c, pr, nodes, &stats)) return s;
  MlpWork w;
  if (slm_status s = proposal_work(c, A, &w)) return s;
  CK(launch(c, SLM_K_PROPOSAL, 0.0,
            [&] { return launch_mlp_forward(c->prop->m, stats, A, w, c->stream); }));
  CK(launch(c, SLM_K_SWARM_INIT, 0.0, [&] {
    return launch_swarm_seed_init(pr, sw, ws_ptr<NodeDesc>(c, S_NODES), A, co, w.O, c->stream);
  }));
  return SLM_OK;
}

// Projection tiles of a search's FP32 pass: forced, fixed, cached for the
// shape (d, padded P, whether base rows can be gathered, log2 of the row
// tiles), or tuned now: every candidate (particles per group 8 / 16 / 24 / 32
// / 48 dividing Pp, x 1 or 2 CTAs per SM, x rows from the level copy or
// gathered from the base rows when the forest keeps them) projects the
// batch's current positions (once to warm, then twice between events) and
// the fastest is kept for the shape. The candidates
// compute the same z and ranges (each z is the same sequence of fused
// multiply-adds), so the extra passes change nothing the search reads.
slm_status pick_tiles(slm_ctx* c, const Problem& pr, const Swarm& sw, int n_tiles, int A,
                      slm_ctx::Tiles* out) {
  if (c->forced.pg) {
    if (!project_group_ok(pr, c->forced.pg))
      return fail(c, SLM_EINVAL, "forced particle group does not divide the padded swarm");
    *out = c->forced;
    return SLM_OK;
  }
  *out = slm_ctx::Tiles{};
  if (!c->tune || n_tiles <= 0) return SLM_OK;
  int lg = 0;
  while ((1 << lg) < n_tiles) ++lg;
  const bool can_gather = pr.Xg && pr.gidx;
  const uint64_t key = ((uint64_t)pr.d << 40) | ((uint64_t)pr.Pp << 16) |
                       ((uint64_t)can_gather << 15) | ((uint64_t)c->tma << 14) | (uint64_t)lg;
  auto it = c->tuned.find(key);
  if (it != c->tuned.end()) {
    *out = it->second;
    return SLM_OK;
  }
  const WorkTile* dt = ws_ptr<WorkTile>(c, S_TILES);
  cudaEvent_t e0 = take_event(c), e1 = take_event(c);
  if (!e0 || !e1) return fail(c, SLM_ECUDA, "cudaEventCreate");
  float best = 0.f;
  slm_ctx::Tiles pick{};
  bool have = false;
  slm_status s = SLM_OK;
  for (int pg : {8, 16, 24, 32, 48}) {
    if (!project_group_ok(pr, pg)) continue;
    // CTAs per SM x row source (entry-ordered copy staged by tensor maps or
    // per-thread copies; gathered rows, per-thread copies)
    for (int v = 0; v < (can_gather ? 6 : 4) && !s; ++v) {
      const int cps = 1 + (v & 1);
      const bool gather = v >= 4;
      const bool tma = v < 2;
      if (tma && !c->tma) continue;
      cudaError_t e = cudaSuccess;
      for (int r = 0; r < 3 && !e; ++r) {
        if (r == 1) e = cudaEventRecord(e0, c->stream);
        if (!e)
          e = launch_project(pr, sw, dt, n_tiles, cps * c->n_sm, c->stream, pg, gather,
                             tma ? A : 0);
        c->launches += 1;
      }
      if (!e) e = cudaEventRecord(e1, c->stream);
      if (!e) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e) {
        s = cuda_fail(c, e, "projection tile tuning");
        break;
      }
      if (!have || ms < best) {
        best = ms;
        pick = slm_ctx::Tiles{pg, cps, ms, gather, tma};
        have = true;
      }
    }
  }
  c->free_events.push_back(e0);
  c->free_events.push_back(e1);
  if (s) return s;
  c->tuned[key] = pick;
  *out = pick;
  return SLM_OK;
}

constexpr size_t kMaxGraphs = 64;  // executable graphs kept per context

// Launch signature of a captured graph: per node in the graph's order, its
// type and, for kernels, function, grid, block, dynamic shared memory and
// cluster shape. Executables are only updated in place from a capture with
// the same signature, so an update changes kernel arguments and nothing else.
cudaError_t graph_signature(cudaGraph_t g, std::vector<uint64_t>* sig) {
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
  if (e) return e;
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && (e = cudaGraphGetNodes(g, nodes.data(), &n))) return e;
  sig->clear();
  sig->reserve(6 * n + 1);
  sig->push_back(n);
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    if ((e = cudaGraphNodeGetType(nd, &ty))) return e;
    sig->push_back((uint64_t)ty);
    if (ty != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp{};
    if ((e = cudaGraphKernelNodeGetParams(nd, &kp))) return e;
    cudaLaunchAttributeValue cl{};
    if ((e = cudaGraphKernelNodeGetAttribute(nd, cudaLaunchAttributeClusterDimension, &cl)))
      return e;
    sig->push_back((uint64_t)(uintptr_t)kp.func);
    sig->push_back(((uint64_t)kp.gridDim.x << 32) | ((uint64_t)kp.gridDim.y << 16) |
                   kp.gridDim.z);
    sig->push_back(((uint64_t)kp.blockDim.x << 32) | ((uint64_t)kp.blockDim.y << 16) |
                   kp.blockDim.z);
    sig->push_back(((uint64_t)kp.sharedMemBytes << 24) | ((uint64_t)cl.clusterDim.x << 16) |
                   ((uint64_t)cl.clusterDim.y << 8) | cl.clusterDim.z);
  }
  return cudaSuccess;
}

// CTAs per (node, particle) of the cluster histogram kernel for a search's
// FP32 pass: the one-wave rule of hist_split (tuning off), cached for the
// shape (criterion, bins, classes, particles, multiplicities, log2 of the
// largest node and of the node count), or tuned now: for every cluster size
// the device can schedule (1..16, slices of at least 256 entries) the
// batch is projected once with the search's tiles and histogrammed once
// between events; the fastest is kept. The histogram pass only reads the
// projections and writes scores and reset ranges, which the search's first
// iteration recomputes, so the extra passes change nothing it reads.
slm_status check_kernel_errors(slm_ctx* c);

slm_status pick_split(slm_ctx* c, const Problem& pr, const Swarm& sw,
                      const std::vector<NodeDesc>& nodes, int n_tiles,
                      const slm_ctx::Tiles& tl, int* S_out, const ClsPlan* cp = nullptr) {
  const bool cls = cp && cp->on;
  int64_t max_len = 0;
  for (const NodeDesc& nd : nodes) max_len = std::max<int64_t>(max_len, nd.seg_len);
  *S_out = cls ? hist_cls_split(pr, (int)nodes.size(), max_len, c->n_sm)
               : batch_split(c, pr, nodes);
  if (!c->tune || nodes.empty() || n_tiles <= 0) return SLM_OK;
  auto lg = [](int64_t v) {
    int l = 0;
    while ((1LL << l) < v) ++l;
    return (int64_t)l;
  };
  const std::vector<int64_t> key{pr.crit, pr.B, pr.K, pr.P, pr.w != nullptr, lg(max_len),
                                 lg((int64_t)nodes.size()), cls ? 1 : 0};
  auto it = c->tuned_split.find(key);
  if (it != c->tuned_split.end()) {
    *S_out = it->second.S;
    return SLM_OK;
  }
  const int A = (int)nodes.size();
  const int smax = cls ? 16 : std::min(16, hist_max_cluster(pr));
  const WorkTile* dt = ws_ptr<WorkTile>(c, S_TILES);
  const NodeDesc* dn = ws_ptr<NodeDesc>(c, S_NODES);
  cudaEvent_t e0 = take_event(c), e1 = take_event(c);
  if (!e0 || !e1) return fail(c, SLM_ECUDA, "cudaEventCreate");
  slm_ctx::Split best{*S_out, 0.f};
  bool have = false;
  for (int S = 1; S <= smax; ++S) {
    if (S > 1 && max_len / S < 256) break;
    if (cls && (S & (S - 1))) continue;  // powers of two
    float ms_min = 0.f;
    bool ok = true;
    for (int r = 0; r < 2 && ok; ++r) {
      cudaError_t e = launch_project(pr, sw, dt, n_tiles, tl.cps * c->n_sm, c->stream, tl.pg,
                                     tl.gather, c->tma && tl.tma ? A : 0);
      if (!e) e = cudaEventRecord(e0, c->stream);
      if (!e)
        e = cls ? launch_hist_cls(pr, sw, dn, A, S, 0, 0, cp->xtab, c->stream)
                : launch_hist_scan(pr, sw, dn, A, S, nullptr, 0, 0, c->stream);
      if (!e) e = cudaEventRecord(e1, c->stream);
      if (!e) e = cudaEventSynchronize(e1);
      c->launches += 2;
      float ms = 0.f;
      if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e) {  // a cluster size the device cannot place: skip it
        (void)cudaGetLastError();
        ok = false;
        break;
      }
      ms_min = r == 0 ? ms : std::min(ms_min, ms);
    }
    if (!ok) continue;
    if (!have || ms_min < best.ms) {
      best = slm_ctx::Split{S, ms_min};
      have = true;
    }
  }
  c->free_events.push_back(e0);
  c->free_events.push_back(e1);
  if (slm_status s = check_kernel_errors(c)) return s;
  c->tuned_split[key] = best;
  *S_out = best.S;
  return SLM_OK;
}

// The T + 1 scoring passes of a search (Algorithm 1's loop). With graphs on
// (and per-launch profiling off) the passes run as one CUDA graph launch: the
// device runs the whole loop of a level without waiting on the host. The
// context keeps executable graphs: one recorded from the same launch inputs
// (`key`: every field of the problem, swarm, plan and tiles, and the buffers
// the launches read) is launched again as it is; otherwise the passes are
// recorded, and an executable with the same launch signature is updated in
// place (kernel arguments only), or a new one is instantiated.
template <class F>
slm_status run_iterations(slm_ctx* c, int T, const std::string& key, F&& pass) {
  if (!c->graphs || c->prof) {
    for (int t = 0; t <= T; ++t)
      if (slm_status s = pass(t)) return s;
    return SLM_OK;
  }
  for (slm_ctx::GraphEntry& ge : c->graph_cache)
    if (ge.key == key) {
      CK(cudaGraphLaunch(ge.exec, c->stream));
      c->launches += ge.launches;
      for (int k = 0; k < SLM_K_COUNT; ++k) {
        c->k_launches[k] += ge.k_launches[k];
        c->k_pairs[k] += ge.k_pairs[k];
      }
      c->graph_launches += 1;
      c->graph_reuses += 1;
      return SLM_OK;
    }
  if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  // the passes are recorded on the context's own stream (recording runs
  // nothing) and the graph is launched on the caller's stream
  slm_ctx::GraphEntry rec;
  rec.key = key;
  rec.launches = c->launches;
  for (int k = 0; k < SLM_K_COUNT; ++k) {
    rec.k_launches[k] = c->k_launches[k];
    rec.k_pairs[k] = c->k_pairs[k];
  }
  const cudaStream_t user = c->stream;
  CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  c->stream = c->cap_stream;
  slm_status s = SLM_OK;
  for (int t = 0; t <= T && !s; ++t) s = pass(t);
  c->stream = user;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (s || e) {
    if (g) cudaGraphDestroy(g);
    return s ? s : cuda_fail(c, e, "cudaStreamEndCapture");
  }
  rec.launches = c->launches - rec.launches;
  for (int k = 0; k < SLM_K_COUNT; ++k) {
    rec.k_launches[k] = c->k_launches[k] - rec.k_launches[k];
    rec.k_pairs[k] = c->k_pairs[k] - rec.k_pairs[k];
  }
  cudaError_t ei = graph_signature(g, &rec.sig);
  slm_ctx::GraphEntry* hit = nullptr;
  if (!ei)
    for (slm_ctx::GraphEntry& ge : c->graph_cache)
      if (ge.sig == rec.sig) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(ge.exec, g, &info) == cudaSuccess) {
          rec.exec = ge.exec;
          ge = std::move(rec);
          hit = &ge;
        } else {
          (void)cudaGetLastError();
        }
        break;
      }
  if (!ei && !hit) {
    if (c->graph_cache.size() >= kMaxGraphs) {
      cudaGraphExecDestroy(c->graph_cache.front().exec);  // freed after in-flight launches
      c->graph_cache.erase(c->graph_cache.begin());
    }
    for (size_t i = 0; i < c->graph_cache.size(); ++i)  // a failed update's entry
      if (c->graph_cache[i].sig == rec.sig) {
        cudaGraphExecDestroy(c->graph_cache[i].exec);
        c->graph_cache.erase(c->graph_cache.begin() + (long)i);
        break;
      }
    ei = cudaGraphInstantiate(&rec.exec, g, 0);
    if (!ei) {
      c->graph_cache.push_back(std::move(rec));
      hit = &c->graph_cache.back();
      c->graph_instantiations += 1;
    }
  } else if (hit) {
    c->graph_updates += 1;
  }
  cudaGraphDestroy(g);
  if (ei) return cuda_fail(c, ei, "graph instantiation");
  c->graph_launches += 1;
  CK(cudaGraphLaunch(hit->exec, c->stream));
  return SLM_OK;
}

// Appends the raw bytes of scalars and pointers: the launch inputs of a
// search, compared whole to find a graph recorded from the same inputs.
struct KeyWriter {
  std::string b;
  template <class T>
  void put(const T& v) {
    static_assert(std::is_arithmetic<T>::value || std::is_pointer<T>::value, "scalar");
    b.append(reinterpret_cast<const char*>(&v), sizeof(T));
  }
  void problem(const Problem& p) {
    put(p.X); put(p.Xg); put(p.gidx); put(p.lab); put(p.y); put(p.w); put(p.E); put(p.Ez);
    put(p.d); put(p.crit); put(p.K); put(p.B); put(p.min_leaf); put(p.P); put(p.Pp);
    put(p.G); put(p.Xb); put(p.dp); put(p.m1); put(p.m2); put(p.mscale);
  }
  void swarm(const Swarm& w) {
    put(w.pos); put(w.vel); put(w.pbest); put(w.gbest); put(w.cur); put(w.pb); put(w.gb);
    put(w.gpart); put(w.giter); put(w.trace); put(w.zmm); put(w.z); put(w.done); put(w.err);
    put(w.T); put(w.sel); put(w.k); put(w.tk_sel); put(w.tk_inv); put(w.tk_pos);
    put(w.tk_k); put(w.tk_kp); put(w.posb); put(w.apso); put(w.ic); put(w.s2);
    put(w.co.inertia); put(w.co.c1); put(w.co.c2); put(w.co.seed); put(w.node_step);
    put(w.n_nodes); put(w.imp);
  }
};

// PSO search of every node of a batch (Algorithm 1, synchronous updates).
slm_status prescreen_search(slm_ctx* c, const slm_params* p, Problem& pr,
                            const std::vector<NodeDesc>& nodes, bool want_trace,
                            Swarm* sw_out);
slm_status check_kernel_errors(slm_ctx* c);

slm_status run_search(slm_ctx* c, const slm_params* p, Problem& pr_in,
                      const std::vector<NodeDesc>& nodes, bool want_trace,
                      Swarm* sw_out) {
  if (p->top_n > 0 && p->top_n < pr_in.d)
    return prescreen_search(c, p, pr_in, nodes, want_trace, sw_out);
  // adaptive PSO scores one more slot per node, its elite candidate (slot
  // P): pr is the evaluation's problem, psw the swarm kernels' (same layout)
  Problem pr = pr_in;
  if (p->apso) {
    pr.P = pr_in.P + 1;
    pr.Pp = (pr.P + kPG - 1) / kPG * kPG;
    pr.G = pr.Pp / kPG;
  }
  const int A = (int)nodes.size();
  // classification nodes (FP32 form) whose rows fit in shared memory run
  // their whole search in one persistent launch; the others (`in`) run the
  // per-iteration kernels, beside it on the context's second stream
  std::vector<char> resident(A, 0);
  int n_res = 0;
  size_t smax = 0;
  int S_res = 1;  // CTAs per resident node
  if (c->node_search && p->proj != SLM_PROJ_BF16_TOPK && p->criterion != SLM_MSE && !p->apso) {
    // candidates: rows and the swarm share fit with the node spread widest;
    // then CTAs per node, up to one particle per warp while the GPU has
    // room; then the nodes that fit at that spread
    const int want = std::min(8, (pr.P + 7) / 8);
    int n_cand = 0;
    for (int a = 0; a < A; ++a)
      n_cand += node_search_smem(pr, nodes[a].seg_len, want) <= kNodeSearchMaxSmem;
    while (S_res * 2 <= want && (int64_t)n_cand * S_res * 2 <= c->n_sm) S_res *= 2;
    for (int a = 0; n_cand > 0 && a < A; ++a) {
      const size_t sm = node_search_smem(pr, nodes[a].seg_len, S_res);
      if (sm <= kNodeSearchMaxSmem) {
        resident[a] = 1;
        ++n_res;
        smax = std::max(smax, sm);
      }
    }
  }
  std::vector<char> in;
  if (n_res > 0 && n_res < A) {
    in.resize(A);
    for (int a = 0; a < A; ++a) in[a] = !resident[a];
  }
  std::vector<WorkTile> tiles;
  double pairs = 0.0, pairs_res = 0.0;
  for (int a = 0; a < A; ++a) {
    const double np = (double)nodes[a].seg_len * pr.P;
    if (resident[a]) {
      pairs_res += np;
      continue;
    }
    pairs += np;
    for (int r = 0; r < nodes[a].seg_len; r += kTS)
      tiles.push_back(WorkTile{a, nodes[a].seg_start + r, std::min(kTS, nodes[a].seg_len - r), 0});
  }
  Swarm sw;
  slm_status s = setup_swarm(c, pr, A, p->n_iters, want_trace, nodes, tiles, &sw);
  if (s) return s;
  // the scoring set-up's per-batch fields (MSE moments) go back to the caller
  pr_in.m1 = pr.m1;
  pr_in.m2 = pr.m2;
  pr_in.mscale = pr.mscale;
  Problem psw = pr;
  psw.P = pr_in.P;
  sw.apso = p->apso ? ws_ptr<ApsoState>(c, S_APSO) : nullptr;
  const SwarmCoef co{p->inertia, p->c1, p->c2, p->seed};
  const NodeDesc* dn = ws_ptr<NodeDesc>(c, S_NODES);
  Bf16Plan bp;
  if (p->proj == SLM_PROJ_BF16_TOPK &&
      (s = setup_bf16(c, pr, nodes, std::min(p->topk, p->n_particles), true, &sw, &bp)))
    return s;
  if (bp.on && bp.k > 0 && c->class_hist && hist_cls_ok(pr) && hist_cls_ok(bp.pr_k)) {
    int64_t len = 0;
    for (const NodeDesc& nd : nodes) len = std::max<int64_t>(len, nd.seg_len);
    if (hist_cls_fits(pr, len)) {
      CK(prepare_hist_cls(bp.pr_k));  // (shared-memory limits are only raised)
      CK(prepare_hist_cls(pr));
      bp.fast = true;
      if (pr.crit == SLM_ENTROPY) bp.xtab = xlogx_table(c->device);
      bp.S_fast = hist_cls_split(pr, A, len, c->n_sm);
      bp.S_fast_k = hist_cls_split(bp.pr_k, A, len, c->n_sm);
    }
  }
  if (p->seeded) {
    if ((s = seed_swarms(c, psw, nodes, sw, co))) return s;
  } else {
    CK(launch(c, SLM_K_SWARM_INIT, 0.0,
              [&] { return launch_swarm_init(psw, sw, dn, A, co, c->stream); }));
  }
  c->last_node_search = 0;
  bool joined = true;
  if (n_res > 0) {
    const int S = S_res;
    std::vector<int32_t> lst;
    for (int a = 0; a < A; ++a)
      if (resident[a]) lst.push_back(a);
    CK(ensure(c->ws[S_NLIST], sizeof(int32_t) * lst.size()));
    CK(cudaMemcpyAsync(c->ws[S_NLIST].p, lst.data(), sizeof(int32_t) * lst.size(),
                       cudaMemcpyHostToDevice, c->stream));
    const int32_t* dl = static_cast<const int32_t*>(c->ws[S_NLIST].p);
    cudaStream_t st = c->stream;
    if (n_res < A && !c->prof) {  // overlap with the per-iteration kernels
      if (!c->side) CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
      if (!c->ev_fork) CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
      if (!c->ev_join) CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
      CK(cudaEventRecord(c->ev_fork, c->stream));
      CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
      st = c->side;
      joined = false;
    }
    CK(launch(c, SLM_K_NODE_SEARCH, pairs_res * (p->n_iters + 1), [&] {
      return launch_node_search(pr, sw, dn, dl, (int)lst.size(), A, S, smax, co, st);
    }));
    if (!joined) CK(cudaEventRecord(c->ev_join, st));
    c->last_node_search = S;
  }
  // plain FP32 searches of whole batches: the move folded into the projection
  StepPlan stp;
  if (n_res == 0 && c->fused_step && !c->forced.pg && !bp.on && !p->apso && step_ok(pr)) {
    bool every = true;
    for (int a = 0; a < A; ++a) every = every && nodes[a].seg_len > 0;
    auto units = [&](int rows) {
      int64_t u = 0;
      for (int a = 0; a < A; ++a) u += (nodes[a].seg_len + rows - 1) / rows;
      return u;
    };
    // a unit of half the particles costs half the rows' work
    // Tile shape: the least estimated time per CTA, units per CTA x (rows
    // per unit + a unit's fixed cost, about kStepUnitRows rows' worth:
    // staging, z stores, range reductions), larger row tiles on ties; a
    // short node is spread over more CTAs by smaller tiles. Every shape gives
    // the same z (the same fused multiply-adds per z).
    int sh = 0, grid = 0, best_tie = 0;
    int64_t best = -1;
    const int want = c->step_shape >= 0 && step_rows(pr, c->step_shape) <= 0 ? 0 : c->step_shape;
    for (int k = 0; k < kStepShapeCount; ++k) {
      const int rows = step_rows(pr, k);
      if (rows <= 0 || (want >= 0 && k != want)) continue;
      CK(prepare_step_kernels(pr, k));
      const int g = step_grid(pr, k, c->n_sm);
      if (g <= 0) continue;
      const int sl = step_slices(pr, k);
      const int64_t u = units(rows) * sl, runs = (u + g - 1) / g;
      const int64_t per = runs * (rows / sl + kStepUnitRows);
      // equal estimates: where every CTA takes one unit, the half-swarm
      // units (each CTA moves half the particles); else the larger tiles
      const int tie = runs == 1 ? (sl > 1 ? 0 : 1) : (sl > 1 ? 1 : 0);
      if (best < 0 || per < best || (per == best && tie < best_tie)) {
        best = per;
        best_tie = tie;
        sh = k;
        grid = g;
      }
    }
    const int rows = step_rows(pr, sh), slices = step_slices(pr, sh);
    std::vector<WorkTile> st;
    if (grid > 0)
      for (int a = 0; a < A; ++a)
        for (int q = 0; q < slices; ++q)
          for (int r = 0; r < nodes[a].seg_len; r += rows)
            st.push_back(WorkTile{a, nodes[a].seg_start + r, std::min(rows, nodes[a].seg_len - r),
                                  q * (pr.Pp / slices)});
    // Folding pays where the chain is latency-bound: a level whose
    // projection is a few waves of units (a tree's levels of one or a few
    // large nodes). Long projections (many nodes, or one very large node)
    // keep the tuned projection and the separate move, where each row tile
    // is not paired with the re-formed positions of its node. Measured in
    // waves of the largest tile shape.
    const int g0 = step_grid(pr, 0, c->n_sm);
    const bool short_level = g0 > 0 && units(step_rows(pr, 0)) <= (int64_t)kFusedMaxWaves * g0;
    if (every && grid > 0 && !st.empty() && (c->fused_step == 2 || short_level)) {
      const size_t apd = (size_t)A * pr.Pp * pr.d;
      CK(ensure(c->ws[S_POS2], sizeof(float) * apd));
      CK(ensure(c->ws[S_IC], sizeof(float) * apd));
      CK(ensure(c->ws[S_S2], sizeof(float) * apd));
      CK(ensure(c->ws[S_STILES], sizeof(WorkTile) * st.size()));
      CK(ensure(c->ws[S_IMP], sizeof(int32_t) * 2 * (size_t)A));
      CK(cudaMemsetAsync(c->ws[S_IMP].p, 0, sizeof(int32_t) * 2 * (size_t)A, c->stream));
      CK(cudaMemcpyAsync(c->ws[S_STILES].p, st.data(), sizeof(WorkTile) * st.size(),
                         cudaMemcpyHostToDevice, c->stream));
      stp.on = true;
      stp.pos[0] = sw.pos;
      stp.pos[1] = ws_ptr<float>(c, S_POS2);
      stp.tiles = ws_ptr<WorkTile>(c, S_STILES);
      stp.n_tiles = (int)st.size();
      stp.grid = grid;
      stp.sh = sh;
      c->last_step_shape = sh;
      sw.ic = ws_ptr<float>(c, S_IC);
      sw.s2 = ws_ptr<float>(c, S_S2);
      sw.co = co;
      sw.imp = ws_ptr<int32_t>(c, S_IMP);
      sw.n_nodes = A;
      c->fused_searches += 1;
    }
  }
  if (n_res < A) {
    int S = batch_split(c, pr, nodes);
    slm_ctx::Tiles tl{};
    if (!bp.on && !stp.on && (s = pick_tiles(c, pr, sw, (int)tiles.size(), A, &tl))) return s;
    HistPlan hp;
    if (!bp.on && (s = setup_hist_plan(c, pr, nodes, in, &hp))) return s;
    ClsPlan cp;
    int64_t max_len = 0;
    for (const NodeDesc& nd : nodes) max_len = std::max<int64_t>(max_len, nd.seg_len);
    if (c->class_hist && !bp.on && hist_cls_ok(pr) && hist_cls_fits(pr, max_len)) {
      CK(prepare_hist_cls(pr));
      cp.on = true;
      cp.xtab = xlogx_table(c->device);
      if (hp.on && hp.n_large)
        cp.S_large = hist_cls_split(pr, hp.n_large, hp.max_large, c->n_sm);
    }
    if (!bp.on && !hp.on &&
        (s = pick_split(c, pr, sw, nodes, (int)tiles.size(), tl, &S, cp.on ? &cp : nullptr)))
      return s;
    cp.S = S;
    // every node scored by k_hist_cls: its last CTA per node takes the gbest
    // step and moves the swarm
    if (stp.on && cp.on && !hp.on && c->node_step && pr.crit != SLM_MSE) sw.node_step = 1;
    c->last_split = S;
    c->cur = tl;
    c->last = tl;
    std::string key;
    if (c->graphs && !c->prof) {
      KeyWriter kw;
      kw.problem(pr);
      kw.swarm(sw);
      kw.put(A); kw.put((int)tiles.size()); kw.put(S); kw.put(p->n_iters); kw.put(c->n_sm);
      kw.put(co.inertia); kw.put(co.c1); kw.put(co.c2); kw.put(co.seed);
      kw.put(tl.pg); kw.put(tl.cps); kw.put(tl.gather); kw.put(tl.tma); kw.put(c->tma);
      kw.put(pairs);
      kw.put(dn); kw.put(ws_ptr<WorkTile>(c, S_TILES)); kw.put(ws_ptr<WorkTile>(c, S_MTILES));
      kw.put(bp.on); kw.put(bp.k); kw.put(bp.kp); kw.put(bp.n_mtiles); kw.put(bp.grid);
      kw.put(bp.S_k); kw.put(bp.pairs_k); kw.put(bp.posb); kw.put(bp.sel); kw.put(bp.inv);
      kw.put(bp.fast); kw.put(bp.S_fast); kw.put(bp.S_fast_k); kw.put(bp.xtab);
      kw.put(hp.on); kw.put(hp.large); kw.put(hp.n_large); kw.put(hp.S_large);
      kw.put(hp.pairs_large); kw.put(hp.small); kw.put(hp.n_small); kw.put(hp.pairs_small);
      kw.put(hp.moved); kw.put(hp.n_moved);
      kw.put(stp.on); kw.put(stp.pos[1]); kw.put(stp.tiles); kw.put(stp.n_tiles);
      kw.put(stp.grid); kw.put(cp.on); kw.put(cp.S); kw.put(cp.S_large); kw.put(cp.xtab);
      if (bp.on) {
        kw.problem(bp.pr_k);
        kw.swarm(bp.sw_k);
      }
      key = std::move(kw.b);
    }
    s = run_iterations(c, p->n_iters, key, [&](int t) {
      return score_batch(c, pr, sw, nodes, (int)tiles.size(), pairs, nullptr, t, &co, S, &bp,
                         &hp, &stp, &cp);
    });
    c->cur = slm_ctx::Tiles{};
    if (!joined) {
      const cudaError_t e = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
      if (!s && e) s = cuda_fail(c, e, "joining the persistent search");
    }
    if (s) return s;
  }
  sw.gb += (size_t)(p->n_iters & 1) * A;  // the final gbest scores
  *sw_out = sw;
  return SLM_OK;
}

// Host twin of the device ranking: a strictly better score (Gini: the exact
// rational Q, larger is better; otherwise the loss), invalid scores last.
bool better_host(const EvalRes& a, const EvalRes& b, int crit) {
  if (!a.valid) return false;
  if (!b.valid) return true;
  if (crit == SLM_GINI)
    return (unsigned __int128)a.num * b.den > (unsigned __int128)b.num * a.den;
  return a.loss < b.loss;
}

// Feature pre-screen (Sec. III-B, Algorithm 2): every feature of every node
// scored on its own in one batched pass (the unit vectors e_k as particles,
// so z = x_k), the top_n best kept per node (stable order: ties to the lower
// feature; then increasing feature order), their columns gathered, the
// swarm search run on that subspace, and gB lifted back to d features.
slm_status prescreen_search(slm_ctx* c, const slm_params* p, Problem& pr,
                            const std::vector<NodeDesc>& nodes, bool want_trace,
                            Swarm* sw_out) {
  const int A = (int)nodes.size(), d = pr.d, n = p->top_n;
  Problem pu = pr;
  pu.P = d;
  pu.Pp = (d + kPG - 1) / kPG * kPG;
  pu.G = pu.Pp / kPG;
  const std::vector<WorkTile> tiles = plan_tiles(nodes);
  Swarm su{};
  if (slm_status s = setup_scoring(c, pu, A, nodes, tiles, &su)) return s;
  CK(ensure(c->ws[S_FPOS], sizeof(float) * (size_t)A * pu.Pp * d));
  su.pos = ws_ptr<float>(c, S_FPOS);
  CK(launch(c, SLM_K_OTHER, 0.0,
            [&] { return launch_unit_positions(su.pos, A, pu.Pp, d, c->stream); }));
  CK(launch(c, SLM_K_OTHER, 0.0,
            [&] { return launch_range_reset(su.zmm, (int64_t)A * pu.Pp, c->stream); }));
  double pairs = 0.0;
  for (const NodeDesc& nd : nodes) pairs += (double)nd.seg_len * d;
  if (slm_status s = score_batch(c, pu, su, nodes, (int)tiles.size(), pairs, nullptr, 0,
                                 nullptr, batch_split(c, pu, nodes)))
    return s;
  if (slm_status s = check_kernel_errors(c)) return s;
  std::vector<EvalRes> sc((size_t)A * pu.Pp);
  CK(cudaMemcpyAsync(sc.data(), su.cur, sizeof(EvalRes) * sc.size(), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::vector<int32_t> feat((size_t)A * n), order(d);
  for (int a = 0; a < A; ++a) {
    const EvalRes* e = sc.data() + (size_t)a * pu.Pp;
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      return better_host(e[x], e[y], pr.crit);
    });
    std::sort(order.begin(), order.begin() + n);
    std::copy(order.begin(), order.begin() + n, feat.begin() + (size_t)a * n);
  }
  CK(ensure(c->ws[S_FEAT], sizeof(int32_t) * feat.size()));
  CK(cudaMemcpyAsync(c->ws[S_FEAT].p, feat.data(), sizeof(int32_t) * feat.size(),
                     cudaMemcpyHostToDevice, c->stream));
  const int32_t* dfeat = ws_ptr<int32_t>(c, S_FEAT);
  CK(ensure(c->ws[W_XS], sizeof(float) * (size_t)(pr.E > 0 ? pr.E : 1) * n));
  float* xs = ws_ptr<float>(c, W_XS);
  CK(launch(c, SLM_K_GATHER, 0.0, [&] {
    return launch_gather_cols(pr.X, d, dfeat, n, ws_ptr<WorkTile>(c, S_TILES),
                              (int)tiles.size(), xs, c->stream);
  }));
  Problem ps = pr;
  ps.X = xs;
  ps.d = n;
  ps.Xg = nullptr;
  ps.gidx = nullptr;
  ps.Xb = nullptr;
  ps.dp = (n + 15) / 16 * 16;
  slm_params q = *p;
  q.top_n = 0;
  Swarm sw;
  if (slm_status s = run_search(c, &q, ps, nodes, want_trace, &sw)) return s;
  CK(ensure(c->ws[S_GFULL], sizeof(float) * (size_t)A * d));
  float* gfull = ws_ptr<float>(c, S_GFULL);
  CK(launch(c, SLM_K_OTHER, 0.0,
            [&] { return launch_lift(sw.gbest, dfeat, A, n, d, gfull, c->stream); }));
  sw.gbest = gfull;
  *sw_out = sw;
  return SLM_OK;
}

// Kernel error word of the last scoring batch (stream-synchronising).
slm_status check_kernel_errors(slm_ctx* c) {
  int32_t e = 0;
  CK(cudaMemcpyAsync(&e, c->ws[S_ERR].p, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (e == kErrMmaTimeout) return fail(c, SLM_ETIMEOUT, "a tensor-core stage did not complete");
  if (e == kErrCopyTimeout) return fail(c, SLM_ETIMEOUT, "a staged copy did not complete");
  if (e) return fail(c, SLM_ECUDA, "a kernel reported error word " + std::to_string(e));
  return SLM_OK;
}

slm_status read_status(slm_ctx* c, int32_t* out) {
  CK(cudaMemcpyAsync(out, c->ws[S_STATUS].p, sizeof(int32_t), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

slm_status reset_status(slm_ctx* c) {
  CK(ensure(c->ws[S_STATUS], sizeof(int32_t)));
  CK(cudaMemsetAsync(c->ws[S_STATUS].p, 0, sizeof(int32_t), c->stream));
  return SLM_OK;
}

// Validates labels / sample indices on the device.
slm_status validate_inputs(slm_ctx* c, const int32_t* labels, int64_t n, int K,
                           const int32_t* idx, int64_t n_idx) {
  slm_status s = reset_status(c);
  if (s) return s;
  CK(launch(c, SLM_K_OTHER, 0.0, [&] {
    return launch_validate(labels, n, K, idx, idx ? n_idx : 0,
                           ws_ptr<int32_t>(c, S_STATUS), c->stream);
  }));
  int32_t st = 0;
  if ((s = read_status(c, &st))) return s;
  if (st) return fail(c, SLM_EINVAL, "label outside [0, K) or sample index outside [0, n)");
  return SLM_OK;
}

template <typename T>
slm_status copy_out(slm_ctx* c, T* dst, const T* src, size_t count) {
  if (!dst || count == 0) return SLM_OK;
  CK(cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyDefault, c->stream));
  return SLM_OK;
}

}  // namespace

// ============================================================================
extern "C" {

const char* slm_status_string(slm_status s) {
  switch (s) {
    case SLM_OK: return "ok";
    case SLM_EINVAL: return "invalid argument";
    case SLM_ENOMEM: return "out of device memory";
    case SLM_ECUDA: return "CUDA error";
    case SLM_ETIMEOUT: return "device wait timed out";
    case SLM_EUNSUPPORTED: return "unsupported size or mode";
  }
  return "unknown status";
}

slm_status slm_create(slm_ctx** out, int device, void* cuda_stream) {
  if (!out) return SLM_EINVAL;
  *out = nullptr;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
    cudaGetLastError();
    return SLM_EINVAL;
  }
  if (cudaSetDevice(device) != cudaSuccess) return SLM_ECUDA;
  if (ensure_xlogx_table(device) != cudaSuccess) return SLM_ECUDA;
  slm_ctx* c = new (std::nothrow) slm_ctx();
  if (!c) return SLM_ENOMEM;
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  int sms = 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess)
    c->n_sm = sms > 0 ? sms : 1;
  *out = c;
  return SLM_OK;
}

void slm_destroy(slm_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto& b : c->ws) release(b);
  for (auto& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : c->free_events) cudaEventDestroy(e);
  for (auto& ge : c->graph_cache) cudaGraphExecDestroy(ge.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
}

slm_status slm_last_error(slm_ctx* c, char* buf, size_t len) {
  if (!c || !buf || len == 0) return SLM_EINVAL;
  std::snprintf(buf, len, "%s", c->err.c_str());
  return SLM_OK;
}

slm_status slm_swarm_uniforms(slm_ctx* c, uint64_t seed, uint32_t node_uid,
                              uint32_t t, int32_t n_particles, int32_t d,
                              int32_t purpose, float* u) {
  if (!c || !u || n_particles < 1 || d < 1 || purpose < 1 || purpose > 255)
    return fail(c, SLM_EINVAL, "bad arguments to slm_swarm_uniforms");
  CK(cudaSetDevice(c->device));
  const size_t cnt = (size_t)n_particles * d;
  float* dst = u;
  const bool dev = is_device_ptr(u);
  if (!dev) {
    CK(ensure(c->ws[S_OUT], sizeof(float) * cnt));
    dst = ws_ptr<float>(c, S_OUT);
  }
  CK(launch(c, SLM_K_OTHER, 0.0, [&] {
    return launch_swarm_uniforms(seed, node_uid, t, n_particles, d, (uint32_t)purpose, dst,
                                 c->stream);
  }));
  if (!dev) {
    if (slm_status s = copy_out(c, u, dst, cnt)) return s;
  }
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

slm_status slm_bootstrap(slm_ctx* c, uint64_t seed, uint32_t tree_id, int64_t n,
                         uint32_t* w) {
  if (!c || !w || n < 1 || n > INT32_MAX)
    return fail(c, SLM_EINVAL, "bad arguments to slm_bootstrap");
  CK(cudaSetDevice(c->device));
  uint32_t* dst = w;
  const bool dev = is_device_ptr(w);
  if (!dev) {
    CK(ensure(c->ws[S_OUT], sizeof(uint32_t) * n));
    dst = ws_ptr<uint32_t>(c, S_OUT);
  }
  CK(launch(c, SLM_K_OTHER, 0.0,
            [&] { return launch_bootstrap(seed, tree_id, n, dst, c->stream); }));
  if (!dev) {
    if (slm_status s = copy_out(c, w, dst, (size_t)n)) return s;
  }
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

}  // extern "C"

namespace {

// Stages a node given by caller arrays and gathers it into entry order:
// rows X[idx], labels / targets, multiplicities. Fills *pr for P particles.
slm_status prepare_node(slm_ctx* c, const slm_params* p, const float* X, int64_t n,
                        int32_t d, const int32_t* labels, const float* y,
                        const int32_t* sample_idx, const uint32_t* weights,
                        int64_t n_idx, int P, Problem* pr) {
  const float *dX, *dy;
  const int32_t *dlab, *didx;
  const uint32_t* dw;
  slm_status s;
  if ((s = stage_in(c, X, (size_t)n * d, c->ws[W_X], &dX))) return s;
  if ((s = stage_in(c, labels, (size_t)n, c->ws[W_LAB], &dlab))) return s;
  if ((s = stage_in(c, y, (size_t)n, c->ws[W_Y], &dy))) return s;
  // multiplicities are always copied: the kernels read them 16 bytes at a time
  dw = nullptr;
  if (weights && n_idx > 0) {
    CK(ensure(c->ws[W_W], sizeof(uint32_t) * (size_t)(n_idx + 16)));
    CK(cudaMemcpyAsync(c->ws[W_W].p, weights, sizeof(uint32_t) * (size_t)n_idx,
                       cudaMemcpyDefault, c->stream));
    dw = ws_ptr<uint32_t>(c, W_W);
  }
  if (sample_idx) {
    if ((s = stage_in(c, sample_idx, (size_t)n_idx, c->ws[W_IDX], &didx))) return s;
  } else {
    CK(ensure(c->ws[W_IDX], sizeof(int32_t) * n_idx));
    CK(launch(c, SLM_K_OTHER, 0.0,
              [&] { return launch_iota(ws_ptr<int32_t>(c, W_IDX), n_idx, n_idx, 1, c->stream); }));
    didx = ws_ptr<int32_t>(c, W_IDX);
  }
  if ((s = validate_inputs(c, dlab, n, p->n_classes, sample_idx ? didx : nullptr, n_idx)))
    return s;
  CK(ensure(c->ws[W_XL], sizeof(float) * (size_t)n_idx * d));
  CK(ensure(c->ws[W_LABL], sizeof(int32_t) * (size_t)(n_idx + 16)));
  CK(ensure(c->ws[W_YL], sizeof(float) * (size_t)(n_idx + 16)));
  float* Xl = ws_ptr<float>(c, W_XL);
  int32_t* ll = dlab ? ws_ptr<int32_t>(c, W_LABL) : nullptr;
  float* yl = dy ? ws_ptr<float>(c, W_YL) : nullptr;
  CK(launch(c, SLM_K_GATHER, 0.0, [&] {
    return launch_gather(dX, dlab, dy, didx, n_idx, d, Xl, ll, yl, c->stream);
  }));
  *pr = make_problem(p, Xl, d, ll, yl, dw, n_idx, P);
  if (p->proj == SLM_PROJ_BF16_TOPK) {
    // the node's rows once more, as bfloat16 tensor-core operands
    const int dp = round16(d);
    const int64_t nb = std::max<int64_t>(1, (n_idx + kMmaRows - 1) / kMmaRows);
    CK(ensure(c->ws[W_XB], sizeof(uint16_t) * (size_t)nb * kMmaRows * dp));
    uint16_t* xb = ws_ptr<uint16_t>(c, W_XB);
    CK(launch(c, SLM_K_GATHER, 0.0, [&] {
      return launch_to_mma_layout(Xl, n_idx, d, dp, kMmaRows, nb, xb, c->stream);
    }));
    pr->Xb = xb;
    pr->dp = dp;
  }
  return SLM_OK;
}

slm_status check_node_args(slm_ctx* c, const slm_params* p, const float* X, int64_t n,
                           int32_t d, const int32_t* labels, const float* y,
                           const int32_t* sample_idx, int64_t* n_idx, bool swarm) {
  if (slm_status s = check_params(c, p, d, swarm)) return s;
  if (!X || n < 1 || n > INT32_MAX) return fail(c, SLM_EINVAL, "bad X or n");
  if ((p->criterion == SLM_MSE) != (y != nullptr) || (labels != nullptr) == (y != nullptr))
    return fail(c, SLM_EINVAL, "exactly one of labels / y, matching the criterion");
  if (!sample_idx) *n_idx = n;
  if (*n_idx < 0 || *n_idx > INT32_MAX) return fail(c, SLM_EINVAL, "n_idx out of range");
  if (p->criterion == SLM_GINI && *n_idx >= (int64_t(1) << 22))
    return fail(c, SLM_EUNSUPPORTED, "Gini needs fewer than 2^22 samples per node");
  return SLM_OK;
}

}  // namespace

extern "C" {

slm_status slm_evaluate_swarm(slm_ctx* c, const slm_params* p, const float* X,
                              int64_t n, int32_t d, const int32_t* labels,
                              const float* y, const int32_t* sample_idx,
                              const uint32_t* weights, int64_t n_idx,
                              const float* positions, int32_t n_pos,
                              slm_eval* out, int32_t* bins_out) {
  if (!c) return SLM_EINVAL;
  if (slm_status s = check_node_args(c, p, X, n, d, labels, y, sample_idx, &n_idx, false))
    return s;
  if (!positions || n_pos < 1 || n_pos > kMaxParticles || !out)
    return fail(c, SLM_EINVAL, "bad positions / n_pos / out");
  if (p->proj != SLM_PROJ_FP32 && p->proj != SLM_PROJ_BF16_TOPK)
    return fail(c, SLM_EINVAL, "proj must be SLM_PROJ_FP32 or SLM_PROJ_BF16_TOPK");
  if (p->proj == SLM_PROJ_BF16_TOPK) {
    if (p->topk < 0 || p->topk > n_pos) return fail(c, SLM_EINVAL, "topk must be in [0, n_pos]");
    if (slm_status s = check_bf16_size(c, d, n_pos)) return s;
  }
  CK(cudaSetDevice(c->device));
  Problem pr;
  if (slm_status s = prepare_node(c, p, X, n, d, labels, y, sample_idx, weights, n_idx,
                                  n_pos, &pr))
    return s;
  std::vector<NodeDesc> nodes{NodeDesc{0, (int32_t)n_idx, 0u, -1}};
  const std::vector<WorkTile> tiles = plan_tiles(nodes);
  Swarm sw{};
  if (slm_status s = setup_scoring(c, pr, 1, nodes, tiles, &sw)) return s;
  CK(ensure(c->ws[S_POS], sizeof(float) * pr.Pp * d));
  CK(cudaMemsetAsync(c->ws[S_POS].p, 0, sizeof(float) * pr.Pp * d, c->stream));
  CK(cudaMemcpyAsync(c->ws[S_POS].p, positions, sizeof(float) * n_pos * d,
                     cudaMemcpyDefault, c->stream));
  sw.pos = ws_ptr<float>(c, S_POS);
  Bf16Plan bp;
  if (p->proj == SLM_PROJ_BF16_TOPK)
    if (slm_status s = setup_bf16(c, pr, nodes, p->topk, false, &sw, &bp)) return s;
  std::vector<int32_t> zinit(2 * pr.Pp);
  for (int i = 0; i < pr.Pp; ++i) {
    zinit[2 * i] = INT32_MAX;
    zinit[2 * i + 1] = INT32_MIN;
  }
  CK(cudaMemcpyAsync(sw.zmm, zinit.data(), sizeof(int32_t) * zinit.size(),
                     cudaMemcpyHostToDevice, c->stream));
  int32_t* dbins = bins_out;
  const bool bins_dev = bins_out && is_device_ptr(bins_out);
  if (bins_out && !bins_dev) {
    CK(ensure(c->ws[W_BINS], sizeof(int32_t) * (size_t)n_pos * n_idx));
    dbins = ws_ptr<int32_t>(c, W_BINS);
  }
  if (slm_status s = score_batch(c, pr, sw, nodes, (int)tiles.size(),
                                 (double)n_idx * n_pos, dbins, 0, nullptr,
                                 batch_split(c, pr, nodes), &bp))
    return s;
  static_assert(sizeof(slm_eval) == sizeof(EvalRes), "layout");
  if (slm_status s = check_kernel_errors(c)) return s;
  CK(cudaMemcpyAsync(out, sw.cur, sizeof(EvalRes) * n_pos, cudaMemcpyDefault, c->stream));
  if (bins_out && !bins_dev)
    CK(cudaMemcpyAsync(bins_out, dbins, sizeof(int32_t) * (size_t)n_pos * n_idx,
                       cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

slm_status slm_seeded_start(slm_ctx* c, const slm_params* p, const float* X, int64_t n,
                            int32_t d, const int32_t* labels, const float* y,
                            const int32_t* sample_idx, const uint32_t* weights, int64_t n_idx,
                            uint32_t node_uid, float* pos_out) {
  if (!c) return SLM_EINVAL;
  if (slm_status s = check_node_args(c, p, X, n, d, labels, y, sample_idx, &n_idx, true))
    return s;
  if (!pos_out || !p->seeded || !c->prop)
    return fail(c, SLM_EINVAL, "needs pos_out, params.seeded = 1 and a proposal in use");
  CK(cudaSetDevice(c->device));
  Problem pr;
  if (slm_status s = prepare_node(c, p, X, n, d, labels, y, sample_idx, weights, n_idx,
                                  p->n_particles, &pr))
    return s;
  std::vector<NodeDesc> nodes{NodeDesc{0, (int32_t)n_idx, node_uid, -1}};
  const std::vector<WorkTile> tiles = plan_tiles(nodes);
  Swarm sw;
  if (slm_status s = setup_swarm(c, pr, 1, 0, false, nodes, tiles, &sw)) return s;
  const SwarmCoef co{p->inertia, p->c1, p->c2, p->seed};
  if (slm_status s = seed_swarms(c, pr, nodes, sw, co)) return s;
  CK(cudaMemcpyAsync(pos_out, sw.pos, sizeof(float) * (size_t)p->n_particles * d,
                     cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

slm_status slm_node_split(slm_ctx* c, const slm_params* p, const float* X,
                          int64_t n, int32_t d, const int32_t* labels,
                          const float* y, const int32_t* sample_idx,
                          const uint32_t* weights, int64_t n_idx,
                          uint32_t node_uid, float* direction_out,
                          float* gbest_out, slm_split* out, double* trace_out) {
  if (!c) return SLM_EINVAL;
  if (slm_status s = check_node_args(c, p, X, n, d, labels, y, sample_idx, &n_idx, true))
    return s;
  if (!out || !direction_out) return fail(c, SLM_EINVAL, "NULL out or direction_out");
  CK(cudaSetDevice(c->device));
  Problem pr;
  if (slm_status s = prepare_node(c, p, X, n, d, labels, y, sample_idx, weights, n_idx,
                                  p->n_particles, &pr))
    return s;
  std::vector<NodeDesc> nodes{NodeDesc{0, (int32_t)n_idx, node_uid, -1}};
  Swarm sw;
  if (slm_status s = run_search(c, p, pr, nodes, trace_out != nullptr, &sw)) return s;
  if (slm_status s = check_kernel_errors(c)) return s;
  EvalRes gb;
  int32_t part = 0, iter = 0;
  std::vector<float> g(d);
  CK(cudaMemcpyAsync(&gb, sw.gb, sizeof(EvalRes), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&part, sw.gpart, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&iter, sw.giter, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(g.data(), sw.gbest, sizeof(float) * d, cudaMemcpyDeviceToHost,
                     c->stream));
  if (trace_out)
    CK(cudaMemcpyAsync(trace_out, sw.trace, sizeof(double) * (p->n_iters + 1),
                       cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::memcpy(&out->eval, &gb, sizeof(EvalRes));
  out->particle = part;
  out->iter_of_best = iter;
  out->threshold = gb.valid ? gb.zmin + (float)gb.bin / gb.inv_w : 0.0f;
  double nrm = 0.0;
  for (int j = 0; j < d; ++j) nrm += (double)g[j] * g[j];
  nrm = std::sqrt(nrm);
  out->norm = (float)nrm;
  std::vector<float> dir(d);
  for (int j = 0; j < d; ++j) dir[j] = nrm > 0.0 ? (float)(g[j] / nrm) : 0.0f;
  CK(cudaMemcpy(direction_out, dir.data(), sizeof(float) * d, cudaMemcpyDefault));
  if (gbest_out) CK(cudaMemcpy(gbest_out, g.data(), sizeof(float) * d, cudaMemcpyDefault));
  return SLM_OK;
}

// Probabilistic search (Sec. II-B). The candidates are scored like a
// swarm's particles, `batch` at a time, by the same projection and
// histogram kernels; the feature ranking scores the unit vectors the same
// way, up to 256 at a time.
slm_status slm_prob_search(slm_ctx* c, const slm_params* p, const slm_prob* pp, const float* X,
                           int64_t n, int32_t d, const int32_t* labels, const float* y,
                           const int32_t* sample_idx, const uint32_t* weights, int64_t n_idx,
                           uint32_t node_uid, float* direction_out, float* best_out,
                           slm_split* out, double* trace_out, int32_t* rank_feat_out,
                           int32_t* kept_out, int32_t* n_kept_out) {
  if (!c) return SLM_EINVAL;
  if (slm_status s = check_node_args(c, p, X, n, d, labels, y, sample_idx, &n_idx, false))
    return s;
  if (!pp || !out || !direction_out) return fail(c, SLM_EINVAL, "NULL prob, out or direction_out");
  if (p->proj != SLM_PROJ_FP32) return fail(c, SLM_EINVAL, "proj must be SLM_PROJ_FP32");
  const int I = pp->n_candidates;
  if (I < 1 || I > (1 << 20) || (int64_t)I * d > (int64_t(1) << 28))
    return fail(c, SLM_EINVAL, "n_candidates must be in [1, 2^20] with n_candidates * d <= 2^28");
  if (pp->R < 1 || pp->R > kProbMaxR) return fail(c, SLM_EINVAL, "R must be in [1, 64]");
  if (!(pp->gamma > 0.0 && pp->gamma <= 1.0)) return fail(c, SLM_EINVAL, "gamma must be in (0, 1]");
  if (!(pp->alpha0 >= 0.0 && pp->alpha0 <= 100.0) || !(pp->alpha >= 0.0) ||
      !std::isfinite(pp->alpha))
    return fail(c, SLM_EINVAL, "alpha0 must be in [0, 100], alpha finite and >= 0");
  if (pp->batch < 1 || pp->batch > kMaxParticles)
    return fail(c, SLM_EINVAL, "batch must be in [1, 256]");
  if (pp->q < 0 || pp->cos_den < 1 || pp->cos_den > 100 || pp->cos_num < 0 ||
      pp->cos_num > pp->cos_den)
    return fail(c, SLM_EINVAL, "q >= 0 and 0 <= cos_num <= cos_den <= 100, cos_den >= 1");
  CK(cudaSetDevice(c->device));
  const int R = std::min<int>(pp->R, d);
  const int chunk = std::min<int>(d, kMaxParticles);
  const int Pmax = std::max(chunk, (int)pp->batch);
  Problem pr;
  if (slm_status s = prepare_node(c, p, X, n, d, labels, y, sample_idx, weights, n_idx, Pmax,
                                  &pr))
    return s;
  std::vector<NodeDesc> nodes{NodeDesc{0, (int32_t)n_idx, node_uid, -1}};
  const std::vector<WorkTile> tiles = plan_tiles(nodes);
  Swarm su{};
  if (slm_status s = setup_scoring(c, pr, 1, nodes, tiles, &su)) return s;
  CK(ensure(c->ws[S_FPOS], sizeof(float) * (size_t)pr.Pp * d));
  su.pos = ws_ptr<float>(c, S_FPOS);
  // scores rows 0 .. P - 1 of su.pos into su.cur
  auto score = [&](int P) -> slm_status {
    Problem pu = pr;
    pu.P = P;
    pu.Pp = (P + kPG - 1) / kPG * kPG;
    pu.G = pu.Pp / kPG;
    CK(launch(c, SLM_K_OTHER, 0.0,
              [&] { return launch_range_reset(su.zmm, (int64_t)pu.Pp, c->stream); }));
    return score_batch(c, pu, su, nodes, (int)tiles.size(), (double)n_idx * P, nullptr, 0,
                       nullptr, batch_split(c, pu, nodes));
  };
  // rank the features by their own split loss (better first, ties to the
  // lower feature)
  std::vector<EvalRes> fe(d);
  for (int f0 = 0; f0 < d; f0 += chunk) {
    const int cnt = std::min(chunk, d - f0);
    const int Pp = (cnt + kPG - 1) / kPG * kPG;
    CK(launch(c, SLM_K_SWARM_INIT, 0.0,
              [&] { return launch_prob_units(f0, cnt, Pp, d, su.pos, c->stream); }));
    if (slm_status s = score(cnt)) return s;
    CK(cudaMemcpyAsync(fe.data() + f0, su.cur, sizeof(EvalRes) * cnt, cudaMemcpyDeviceToHost,
                       c->stream));
  }
  if (slm_status s = check_kernel_errors(c)) return s;
  CK(cudaStreamSynchronize(c->stream));
  std::vector<int32_t> rank_feat(d);
  std::iota(rank_feat.begin(), rank_feat.end(), 0);
  std::stable_sort(rank_feat.begin(), rank_feat.end(),
                   [&](int a, int b) { return better_host(fe[a], fe[b], pr.crit); });
  // rank weights gamma^r by repeated products (rank r + 1) and coefficient
  // ranges floor(alpha0 exp(-alpha (r + 1)))
  const size_t tab_bytes = sizeof(double) * d + 2 * sizeof(int32_t) * d;
  std::vector<unsigned char> tab(tab_bytes);
  double* w = reinterpret_cast<double*>(tab.data());
  int32_t* m = reinterpret_cast<int32_t*>(tab.data() + sizeof(double) * d);
  int32_t* rf = m + d;
  w[0] = 1.0;
  for (int r = 1; r < d; ++r) w[r] = w[r - 1] * pp->gamma;
  for (int r = 0; r < d; ++r) {
    m[r] = (int32_t)std::floor(pp->alpha0 * std::exp(-pp->alpha * (double)(r + 1)));
    rf[r] = rank_feat[r];
  }
  CK(ensure(c->ws[S_PRTAB], tab_bytes));
  CK(cudaMemcpyAsync(c->ws[S_PRTAB].p, tab.data(), tab_bytes, cudaMemcpyHostToDevice,
                     c->stream));
  const double* dw = ws_ptr<double>(c, S_PRTAB);
  const int32_t* dm = reinterpret_cast<const int32_t*>(dw + d);
  const int32_t* drf = dm + d;
  const int nb = (I + pp->batch - 1) / pp->batch;
  CK(ensure(c->ws[S_PRALL], sizeof(float) * (size_t)I * d));
  CK(ensure(c->ws[S_PRSC], sizeof(EvalRes) * (size_t)I));
  // best score, its index, trace[nb], best vector[d], kept[q], n_kept
  const size_t off_idx = 64, off_trace = 128, off_pos = off_trace + round_up(8 * (size_t)nb, 64),
               off_kept = off_pos + round_up(4 * (size_t)d, 64),
               off_nk = off_kept + round_up(4 * (size_t)std::max(pp->q, 1), 64);
  CK(ensure(c->ws[S_PRBEST], off_nk + 64));
  CK(ensure(c->ws[S_PRUNE], (size_t)I));
  char* bb = static_cast<char*>(c->ws[S_PRBEST].p);
  EvalRes* dbest = reinterpret_cast<EvalRes*>(bb);
  int32_t* dbest_idx = reinterpret_cast<int32_t*>(bb + off_idx);
  double* dtrace = reinterpret_cast<double*>(bb + off_trace);
  float* dbest_pos = reinterpret_cast<float*>(bb + off_pos);
  int32_t* dkept = reinterpret_cast<int32_t*>(bb + off_kept);
  int32_t* dnk = reinterpret_cast<int32_t*>(bb + off_nk);
  float* all_pos = ws_ptr<float>(c, S_PRALL);
  EvalRes* all_sc = ws_ptr<EvalRes>(c, S_PRSC);
  CK(cudaMemsetAsync(dbest_pos, 0, sizeof(float) * d, c->stream));
  CK(launch(c, SLM_K_OTHER, 0.0, [&] { return launch_prob_init(dbest, dbest_idx, c->stream); }));
  for (int b = 0; b < nb; ++b) {
    const int c0 = b * pp->batch, cnt = std::min<int>(pp->batch, I - c0);
    const int Pp = (cnt + kPG - 1) / kPG * kPG;
    CK(launch(c, SLM_K_SWARM_INIT, 0.0, [&] {
      return launch_prob_candidates(p->seed, node_uid, c0, cnt, Pp, d, drf, dw, dm, R, su.pos,
                                    all_pos, c->stream);
    }));
    if (slm_status s = score(cnt)) return s;
    Problem pb = pr;
    pb.P = cnt;
    CK(launch(c, SLM_K_OTHER, 0.0, [&] {
      return launch_prob_best(pb, su.cur, c0, b, dbest, dbest_idx, all_pos, dbest_pos, dtrace,
                              all_sc, c->stream);
    }));
  }
  if (pp->q > 0)
    CK(launch(c, SLM_K_OTHER, 0.0, [&] {
      return launch_prob_prune(pr.crit, I, d, all_pos, all_sc, pp->q, pp->cos_num,
                               pp->cos_den, ws_ptr<uint8_t>(c, S_PRUNE), dkept, dnk,
                               c->stream);
    }));
  else
    CK(cudaMemsetAsync(dnk, 0, sizeof(int32_t), c->stream));
  if (slm_status s = check_kernel_errors(c)) return s;
  EvalRes gb;
  int32_t bidx = 0, nk = 0;
  std::vector<float> g(d);
  CK(cudaMemcpyAsync(&gb, dbest, sizeof(EvalRes), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&bidx, dbest_idx, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&nk, dnk, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(g.data(), dbest_pos, sizeof(float) * d, cudaMemcpyDeviceToHost, c->stream));
  if (trace_out)
    CK(cudaMemcpyAsync(trace_out, dtrace, sizeof(double) * nb, cudaMemcpyDefault, c->stream));
  if (kept_out && pp->q > 0)
    CK(cudaMemcpyAsync(kept_out, dkept, sizeof(int32_t) * pp->q, cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (n_kept_out) *n_kept_out = nk;
  if (rank_feat_out)
    CK(cudaMemcpy(rank_feat_out, rank_feat.data(), sizeof(int32_t) * d, cudaMemcpyDefault));
  std::memcpy(&out->eval, &gb, sizeof(EvalRes));
  out->particle = bidx;
  out->iter_of_best = bidx / pp->batch;
  out->threshold = gb.valid ? gb.zmin + (float)gb.bin / gb.inv_w : 0.0f;
  double nrm = 0.0;
  for (int j = 0; j < d; ++j) nrm += (double)g[j] * g[j];
  nrm = std::sqrt(nrm);
  out->norm = (float)nrm;
  std::vector<float> dir(d);
  for (int j = 0; j < d; ++j) dir[j] = nrm > 0.0 ? (float)(g[j] / nrm) : 0.0f;
  CK(cudaMemcpy(direction_out, dir.data(), sizeof(float) * d, cudaMemcpyDefault));
  if (best_out) CK(cudaMemcpy(best_out, g.data(), sizeof(float) * d, cudaMemcpyDefault));
  return SLM_OK;
}

// ---- forests ------------------------------------------------------------------

static slm_status forest_alloc_trees(slm_ctx* c, slm_forest* f) {
  const size_t TH = (size_t)f->n_trees * f->H;
  const size_t bytes = TH * (4 + 4 * (size_t)f->d + 4 + 4 + 4 + 4 + 8 + 8 + 8 + 8 + 8) + 256;
  CK(ensure(f->tree_mem, bytes));
  unsigned char* p = static_cast<unsigned char*>(f->tree_mem.p);
  auto take = [&](size_t sz) {
    unsigned char* r = p;
    p += (sz + 15) & ~size_t(15);
    return r;
  };
  f->tr.weight = (int64_t*)take(8 * TH);
  f->tr.leaf_value = (double*)take(8 * TH);
  f->tr.loss = (double*)take(8 * TH);
  f->tr.n_left = (int64_t*)take(8 * TH);
  f->tr.n_right = (int64_t*)take(8 * TH);
  f->tr.kind = (int32_t*)take(4 * TH);
  f->tr.zmin = (float*)take(4 * TH);
  f->tr.inv_w = (float*)take(4 * TH);
  f->tr.bin = (int32_t*)take(4 * TH);
  f->tr.leaf_class = (int32_t*)take(4 * TH);
  f->tr.dir = (float*)take(4 * TH * f->d);
  CK(cudaMemsetAsync(f->tree_mem.p, 0, f->tree_mem.cap, c->stream));
  std::vector<int32_t> minus(TH, -1);
  CK(cudaMemcpyAsync(f->tr.kind, minus.data(), 4 * TH, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

void slm_forest_free(slm_forest* f) {
  if (!f) return;
  cudaSetDevice(f->device);
  DevBuf* bufs[] = {&f->own_X, &f->tree_mem, &f->side, &f->lXb};
  for (DevBuf* b : bufs) release(*b);
  for (int i = 0; i < 2; ++i) {
    release(f->lX[i]);
    release(f->lab[i]);
    release(f->ly[i]);
    release(f->lw[i]);
    release(f->lidx[i]);
  }
  delete f;
}

namespace {
// A forest's start (slm_forest_begin). y_per_tree: y holds n_trees target
// vectors of n samples, tree t fitting y[t n .. t n + n) (boosting's class
// trees of one round; no bootstrap); tree t takes the global id id0 + t stride.
slm_status forest_begin_impl(slm_ctx* c, const slm_params* p, const float* X, int64_t n,
                             int32_t d, const int32_t* labels, const float* y, bool y_per_tree,
                             int64_t id0, int64_t stride, slm_forest** out);
}  // namespace

slm_status slm_forest_begin(slm_ctx* c, const slm_params* p, const float* X,
                            int64_t n, int32_t d, const int32_t* labels,
                            const float* y, slm_forest** out) {
  if (!c) return SLM_EINVAL;
  return forest_begin_impl(c, p, X, n, d, labels, y, false, c->tree_id0, c->tree_stride, out);
}

namespace {
slm_status forest_begin_impl(slm_ctx* c, const slm_params* p, const float* X, int64_t n,
                             int32_t d, const int32_t* labels, const float* y, bool y_per_tree,
                             int64_t id0, int64_t stride, slm_forest** out) {
  if (!c || !out) return fail(c, SLM_EINVAL, "NULL context or output");
  *out = nullptr;
  if (slm_status s = check_params(c, p, d, true)) return s;
  if (!X || n < 1 || n > INT32_MAX)
    return fail(c, SLM_EINVAL, "bad X or n");
  if ((p->criterion == SLM_MSE) != (y != nullptr) || (labels != nullptr) == (y != nullptr))
    return fail(c, SLM_EINVAL, "exactly one of labels / y, matching the criterion");
  if (p->max_depth < 0 || p->max_depth > 15)
    return fail(c, SLM_EINVAL, "max_depth must be in [0, 15]");
  if (p->n_trees < 1 || p->n_trees > 65535)
    return fail(c, SLM_EINVAL, "n_trees must be in [1, 65535]");
  if (id0 + (int64_t)(p->n_trees - 1) * stride > 65535)
    return fail(c, SLM_EINVAL, "global tree ids (slm_set_tree_ids) pass 65535");
  if (y_per_tree && (!y || p->bootstrap))
    return fail(c, SLM_EINVAL, "per-tree targets need y and no bootstrap");
  if (p->criterion == SLM_GINI && n >= (int64_t(1) << 22))
    return fail(c, SLM_EUNSUPPORTED, "Gini needs fewer than 2^22 samples per tree");
  if ((int64_t)n * p->n_trees > INT32_MAX)
    return fail(c, SLM_EUNSUPPORTED, "n * n_trees must be < 2^31");
  CK(cudaSetDevice(c->device));
  slm_forest* f = new (std::nothrow) slm_forest();
  if (!f) return fail(c, SLM_ENOMEM, "host allocation failed");
  f->ctx = c;
  f->device = c->device;
  f->params = *p;
  f->tree_id0 = id0;
  f->tree_stride = stride;
  f->n = n;
  f->d = d;
  f->H = (1 << (p->max_depth + 1)) - 1;
  f->n_trees = p->n_trees;
  f->tree_evals.assign((size_t)p->n_trees, 0);
  f->K = p->criterion == SLM_MSE ? 1 : p->n_classes;
  const bool bf16 = p->proj == SLM_PROJ_BF16_TOPK;
  f->align = bf16 ? kMmaRows : 4;
  slm_status s;
  auto bail = [&](slm_status st) {
    slm_forest_free(f);
    return st;
  };
  const float *dX, *dy;
  const int32_t* dlab;
  if ((s = stage_in(c, X, (size_t)n * d, c->ws[W_X], &dX))) return bail(s);
  if ((s = stage_in(c, labels, (size_t)n, c->ws[W_LAB], &dlab))) return bail(s);
  if ((s = stage_in(c, y, (size_t)n * (y_per_tree ? p->n_trees : 1), c->ws[W_Y], &dy)))
    return bail(s);
  if ((s = validate_inputs(c, dlab, n, p->n_classes, nullptr, 0))) return bail(s);
  if ((s = forest_alloc_trees(c, f))) return bail(s);
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device) != cudaSuccess) l2 = 0;
  const size_t xbytes = sizeof(float) * (size_t)n * d;
  if (!bf16 && p->n_trees > 1 && xbytes <= (size_t)l2 / 4) {
    cudaError_t ex = ensure(f->own_X, xbytes);
    if (!ex) ex = cudaMemcpyAsync(f->own_X.p, dX, xbytes, cudaMemcpyDeviceToDevice, c->stream);
    if (ex) return bail(cuda_fail(c, ex, "base rows"));
    f->X = static_cast<const float*>(f->own_X.p);
  }
  f->weighted = p->bootstrap != 0;
  f->level.clear();
  cudaError_t e;
  // root entries of every tree: sample ids (+ multiplicities) in lidx[1] / lw[1]
  int64_t E = 0, ecap = 0;
  const size_t cap = (size_t)n * f->n_trees;
  if ((e = ensure(f->lidx[1], 4 * cap))) return bail(cuda_fail(c, e, "level buffers"));
  if (f->weighted) {
    DevBuf wall, offs, cnts;
    auto cleanup = [&]() {
      release(wall);
      release(offs);
      release(cnts);
    };
    if ((e = ensure(f->lw[1], 4 * cap)) || (e = ensure(wall, 4 * cap)) ||
        (e = ensure(offs, 8 * (size_t)f->n_trees)) || (e = ensure(cnts, 4 * (size_t)f->n_trees))) {
      cleanup();
      return bail(cuda_fail(c, e, "bootstrap buffers"));
    }
    std::vector<int64_t> off(f->n_trees);
    for (int t = 0; t < f->n_trees; ++t) {
      off[t] = (int64_t)t * n;
      c->launches += 1;
      e = launch_bootstrap(p->seed, f->tree_id(t), n, static_cast<uint32_t*>(wall.p) + off[t],
                           c->stream);
      if (e) {
        cleanup();
        return bail(cuda_fail(c, e, "bootstrap"));
      }
    }
    std::vector<int32_t> cnt(f->n_trees);
    c->launches += 1;
    if ((e = cudaMemcpyAsync(offs.p, off.data(), 8 * off.size(), cudaMemcpyHostToDevice,
                             c->stream)) ||
        (e = launch_compact_nonzero(static_cast<uint32_t*>(wall.p), f->n_trees, n,
                                    static_cast<int32_t*>(f->lidx[1].p),
                                    static_cast<uint32_t*>(f->lw[1].p),
                                    static_cast<int64_t*>(offs.p),
                                    static_cast<int32_t*>(cnts.p), c->stream)) ||
        (e = cudaMemcpyAsync(cnt.data(), cnts.p, 4 * cnt.size(), cudaMemcpyDeviceToHost,
                             c->stream)) ||
        (e = cudaStreamSynchronize(c->stream))) {
      cleanup();
      return bail(cuda_fail(c, e, "bootstrap compaction"));
    }
    cleanup();
    for (int t = 0; t < f->n_trees; ++t) E += round_up(cnt[t], f->align);
    ecap = level_capacity(E, f->n_trees, p->max_depth, f->align, p->min_leaf, true);
    if ((e = ensure(f->lidx[0], 4 * (size_t)ecap)) || (e = ensure(f->lw[0], 4 * (size_t)ecap)) ||
        (e = cudaMemsetAsync(f->lidx[0].p, 0, 4 * (size_t)ecap, c->stream)) ||
        (e = cudaMemsetAsync(f->lw[0].p, 0, 4 * (size_t)ecap, c->stream)))
      return bail(cuda_fail(c, e, "level buffers"));
    int64_t pos = 0;
    for (int t = 0; t < f->n_trees; ++t) {
      if ((e = cudaMemcpyAsync(static_cast<int32_t*>(f->lidx[0].p) + pos,
                               static_cast<int32_t*>(f->lidx[1].p) + off[t], 4 * (size_t)cnt[t],
                               cudaMemcpyDeviceToDevice, c->stream)) ||
          (e = cudaMemcpyAsync(static_cast<uint32_t*>(f->lw[0].p) + pos,
                               static_cast<uint32_t*>(f->lw[1].p) + off[t], 4 * (size_t)cnt[t],
                               cudaMemcpyDeviceToDevice, c->stream)))
        return bail(cuda_fail(c, e, "bag packing"));
      f->level.push_back(LevelNode{(int32_t)pos, cnt[t], t * f->H, 0});
      pos += round_up(cnt[t], f->align);
    }
  } else {
    const int64_t n4 = round_up(n, f->align);
    E = n4 * f->n_trees;
    ecap = level_capacity(E, f->n_trees, p->max_depth, f->align, p->min_leaf, false);
    if ((e = ensure(f->lidx[0], 4 * (size_t)ecap)) ||
        (e = cudaMemsetAsync(f->lidx[0].p, 0, 4 * (size_t)ecap, c->stream)))
      return bail(cuda_fail(c, e, "level buffers"));
    c->launches += 1;
    if ((e = launch_iota(static_cast<int32_t*>(f->lidx[0].p), n, n4, f->n_trees, c->stream)))
      return bail(cuda_fail(c, e, "iota"));
    for (int t = 0; t < f->n_trees; ++t)
      f->level.push_back(LevelNode{(int32_t)(t * n4), (int32_t)n, t * f->H, 0});
  }
  // level-resident arrays; every node segment starts at a multiple of 4
  // entries (16 bytes), with room for the padding of a full level
  for (int i = 0; i < 2; ++i) {
    if ((e = ensure(f->lX[i], sizeof(float) * (size_t)ecap * d)) ||
        (e = ensure(f->lidx[i], sizeof(int32_t) * (size_t)ecap)) ||
        (dlab && (e = ensure(f->lab[i], sizeof(int32_t) * (size_t)ecap))) ||
        (dy && (e = ensure(f->ly[i], sizeof(float) * (size_t)ecap))) ||
        (f->weighted && (e = ensure(f->lw[i], sizeof(uint32_t) * (size_t)ecap))))
      return bail(cuda_fail(c, e, "level buffers"));
  }
  for (int i = 0; i < 2; ++i) {  // padding entries hold defined values
    if ((dlab && (e = cudaMemsetAsync(f->lab[i].p, 0, sizeof(int32_t) * (size_t)ecap, c->stream))) ||
        (dy && (e = cudaMemsetAsync(f->ly[i].p, 0, sizeof(float) * (size_t)ecap, c->stream))) ||
        (i == 1 && f->weighted &&
         (e = cudaMemsetAsync(f->lw[i].p, 0, sizeof(uint32_t) * (size_t)ecap, c->stream))))
      return bail(cuda_fail(c, e, "level buffers"));
  }
  if ((e = ensure(f->side, (size_t)ecap))) return bail(cuda_fail(c, e, "level buffers"));
  if (bf16 && (e = ensure(f->lXb, sizeof(uint16_t) * (size_t)round_up(ecap, kMmaRows) *
                                      round16(d))))
    return bail(cuda_fail(c, e, "level buffers"));
  c->launches += 1;
  if ((e = launch_gather(dX, dlab, dy, static_cast<int32_t*>(f->lidx[0].p), ecap, d,
                         static_cast<float*>(f->lX[0].p),
                         dlab ? static_cast<int32_t*>(f->lab[0].p) : nullptr,
                         dy ? static_cast<float*>(f->ly[0].p) : nullptr, c->stream)))
    return bail(cuda_fail(c, e, "root gather"));
  // per-tree targets: tree t's entries (samples 0 .. n - 1 in order, from
  // entry t n4) take its own vector
  const int64_t n4 = round_up(n, f->align);
  for (int t = 1; y_per_tree && t < f->n_trees; ++t)
    if ((e = cudaMemcpyAsync(static_cast<float*>(f->ly[0].p) + t * n4, dy + (int64_t)t * n,
                             sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream)))
      return bail(cuda_fail(c, e, "per-tree targets"));
  if ((e = cudaStreamSynchronize(c->stream))) return bail(cuda_fail(c, e, "root gather"));
  f->cur = 0;
  *out = f;
  return SLM_OK;
}
}  // namespace

slm_status slm_grow_level(slm_ctx* c, slm_forest* f, int32_t* n_split_out) {
  if (!c || !f) return fail(c, SLM_EINVAL, "NULL context or forest");
  if (n_split_out) *n_split_out = 0;
  if (f->done || f->level.empty()) {
    f->done = true;
    return SLM_OK;
  }
  CK(cudaSetDevice(c->device));
  const slm_params* p = &f->params;
  const int L = (int)f->level.size();
  const int K = f->K;
  const int cu = f->cur;
  const bool mse = p->criterion == SLM_MSE;
  int64_t E = 0;
  for (const LevelNode& ln : f->level) E = std::max<int64_t>(E, (int64_t)ln.seg_start + ln.seg_len);
  Problem pr = make_problem(p, static_cast<float*>(f->lX[cu].p), f->d,
                            mse ? nullptr : static_cast<int32_t*>(f->lab[cu].p),
                            mse ? static_cast<float*>(f->ly[cu].p) : nullptr,
                            f->weighted ? static_cast<uint32_t*>(f->lw[cu].p) : nullptr, E,
                            p->n_particles);
  if (f->X) {
    pr.Xg = f->X;
    pr.gidx = static_cast<const int32_t*>(f->lidx[cu].p);
  }

  // 1. statistics and leaf values of every node of the level (per tile)
  std::vector<WorkTile> ltiles;
  std::vector<int32_t> ltile0(L + 1);
  for (int l = 0; l < L; ++l) {
    ltile0[l] = (int32_t)ltiles.size();
    const LevelNode& ln = f->level[l];
    for (int s = 0; s < ln.seg_len; s += kTS)
      ltiles.push_back(WorkTile{l, ln.seg_start + s, std::min(kTS, ln.seg_len - s), 0});
  }
  ltile0[L] = (int32_t)ltiles.size();
  const int n_lt = (int)ltiles.size();
  CK(ensure(c->ws[S_GLVLNODES], sizeof(LevelNode) * L));
  CK(ensure(c->ws[S_GLVLSPLIT], sizeof(int32_t) * L));
  CK(ensure(c->ws[S_GLVLCLS], sizeof(unsigned long long) * (size_t)L * K));
  CK(ensure(c->ws[S_GLVLPAR], sizeof(double) * 2 * (size_t)L));
  CK(ensure(c->ws[S_GLTILES], sizeof(WorkTile) * n_lt));
  CK(ensure(c->ws[S_GLTILE0], sizeof(int32_t) * (L + 1)));
  CK(ensure(c->ws[S_GACCW], sizeof(unsigned long long) * L));
  CK(ensure(c->ws[S_GACCY], sizeof(int32_t) * 2 * L));
  CK(ensure(c->ws[S_GTILESUM], sizeof(double) * 2 * (size_t)n_lt));
  CK(cudaMemcpyAsync(c->ws[S_GLVLNODES].p, f->level.data(), sizeof(LevelNode) * L,
                     cudaMemcpyHostToDevice, c->stream));
  if (n_lt)
    CK(cudaMemcpyAsync(c->ws[S_GLTILES].p, ltiles.data(), sizeof(WorkTile) * n_lt,
                       cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->ws[S_GLTILE0].p, ltile0.data(), sizeof(int32_t) * (L + 1),
                     cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(c->ws[S_GLVLCLS].p, 0, sizeof(unsigned long long) * (size_t)L * K, c->stream));
  CK(cudaMemsetAsync(c->ws[S_GACCW].p, 0, sizeof(unsigned long long) * L, c->stream));
  {
    std::vector<int32_t> yinit(2 * (size_t)L);
    for (int l = 0; l < L; ++l) {
      yinit[l] = INT32_MAX;
      yinit[L + l] = INT32_MIN;
    }
    CK(cudaMemcpyAsync(c->ws[S_GACCY].p, yinit.data(), sizeof(int32_t) * 2 * L,
                       cudaMemcpyHostToDevice, c->stream));
  }
  LevelAcc lacc{static_cast<unsigned long long*>(c->ws[S_GLVLCLS].p),
                static_cast<unsigned long long*>(c->ws[S_GACCW].p), static_cast<int32_t*>(c->ws[S_GACCY].p),
                static_cast<int32_t*>(c->ws[S_GACCY].p) + L, static_cast<double*>(c->ws[S_GTILESUM].p)};
  CK(launch(c, SLM_K_NODE_STATS, 0.0, [&] {
    return launch_node_stats(pr, static_cast<LevelNode*>(c->ws[S_GLVLNODES].p), L,
                             static_cast<WorkTile*>(c->ws[S_GLTILES].p), n_lt,
                             static_cast<int32_t*>(c->ws[S_GLTILE0].p), lacc, f->tr, p->max_depth,
                             static_cast<double*>(c->ws[S_GLVLPAR].p),
                             static_cast<int32_t*>(c->ws[S_GLVLSPLIT].p), c->stream);
  }));
  c->launches += 1;  // the per-node finishing kernel
  std::vector<int32_t> splittable(L);
  CK(cudaMemcpyAsync(splittable.data(), c->ws[S_GLVLSPLIT].p, sizeof(int32_t) * L,
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));

  // 2. swarm search of the splittable nodes, all in one batch
  std::vector<NodeDesc> snodes;
  std::vector<int32_t> smap;
  std::vector<int32_t> stile0;
  int32_t n_st = 0;
  for (int l = 0; l < L; ++l) {
    if (!splittable[l]) continue;
    const LevelNode& ln = f->level[l];
    const int tree = ln.slot / f->H, h = ln.slot % f->H;
    snodes.push_back(NodeDesc{ln.seg_start, ln.seg_len,
                              (f->tree_id(tree) << 16) | (uint32_t)h, ln.slot});
    smap.push_back(l);
    stile0.push_back(n_st);
    n_st += (ln.seg_len + kTS - 1) / kTS;  // the tiles plan_tiles makes
  }
  stile0.push_back(n_st);
  const int A = (int)snodes.size();
  if (A == 0) {
    f->done = true;
    f->level.clear();
    return SLM_OK;
  }
  if (p->proj == SLM_PROJ_BF16_TOPK) {
    // the level's rows as bfloat16 tensor-core operands
    const int dp = round16(f->d);
    const int64_t nb = (E + kMmaRows - 1) / kMmaRows;
    uint16_t* xb = static_cast<uint16_t*>(f->lXb.p);
    CK(launch(c, SLM_K_GATHER, 0.0, [&] {
      return launch_to_mma_layout(pr.X, E, f->d, dp, kMmaRows, nb, xb, c->stream);
    }));
    pr.Xb = xb;
    pr.dp = dp;
  }
  Swarm sw;
  if (slm_status s = run_search(c, p, pr, snodes, false, &sw)) return s;
  if (slm_status s = check_kernel_errors(c)) return s;
  for (const NodeDesc& nd : snodes) {
    const int64_t ev = (int64_t)nd.seg_len * p->n_particles * (p->n_iters + 1);
    f->evaluations += ev;
    f->tree_evals[(size_t)(nd.slot / f->H)] += ev;
  }

  // 3. partition on gB (per tile), zero-gain test and tree fields (per node)
  CK(ensure(c->ws[S_GSMAP], sizeof(int32_t) * A));
  CK(ensure(c->ws[S_GOUT3], sizeof(int32_t) * 3 * A));
  CK(ensure(c->ws[S_GDST], sizeof(int32_t) * 2 * A));
  CK(ensure(c->ws[S_GSTILE0], sizeof(int32_t) * (A + 1)));
  CK(ensure(c->ws[S_GTILELEFT], sizeof(int32_t) * (size_t)n_st));
  CK(ensure(c->ws[S_GTILEBASE], sizeof(int32_t) * (size_t)n_st));
  CK(ensure(c->ws[S_GPLK], sizeof(unsigned long long) * (size_t)A * K));
  CK(ensure(c->ws[S_GPWL], sizeof(unsigned long long) * A));
  CK(cudaMemcpyAsync(c->ws[S_GSMAP].p, smap.data(), sizeof(int32_t) * A, cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaMemcpyAsync(c->ws[S_GSTILE0].p, stile0.data(), sizeof(int32_t) * (A + 1),
                     cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(c->ws[S_GPLK].p, 0, sizeof(unsigned long long) * (size_t)A * K, c->stream));
  CK(cudaMemsetAsync(c->ws[S_GPWL].p, 0, sizeof(unsigned long long) * A, c->stream));
  if (slm_status s = reset_status(c)) return s;
  const NodeDesc* dsn = ws_ptr<NodeDesc>(c, S_NODES);
  // every searched node's tiles (the search uploads only the tiles of the
  // nodes its per-iteration kernels project)
  const std::vector<WorkTile> ptiles = plan_tiles(snodes);
  CK(ensure(c->ws[S_TILES], sizeof(WorkTile) * ptiles.size()));
  if (!ptiles.empty())
    CK(cudaMemcpyAsync(c->ws[S_TILES].p, ptiles.data(), sizeof(WorkTile) * ptiles.size(),
                       cudaMemcpyHostToDevice, c->stream));
  const WorkTile* dst_tiles = ws_ptr<WorkTile>(c, S_TILES);
  PartAcc pacc{static_cast<unsigned long long*>(c->ws[S_GPLK].p),
               static_cast<unsigned long long*>(c->ws[S_GPWL].p)};
  CK(launch(c, SLM_K_PARTITION, 0.0, [&] {
    return launch_partition(pr, sw, dst_tiles, n_st, static_cast<uint8_t*>(f->side.p),
                            static_cast<int32_t*>(c->ws[S_GTILELEFT].p), pacc, c->stream);
  }));
  CK(launch(c, SLM_K_PARTITION, 0.0, [&] {
    return launch_decide(pr, sw, dsn, static_cast<int32_t*>(c->ws[S_GSMAP].p),
                         static_cast<int32_t*>(c->ws[S_GSTILE0].p), A,
                         static_cast<int32_t*>(c->ws[S_GTILELEFT].p),
                         static_cast<int32_t*>(c->ws[S_GTILEBASE].p),
                         static_cast<unsigned long long*>(c->ws[S_GLVLCLS].p),
                         static_cast<double*>(c->ws[S_GLVLPAR].p), pacc, f->tr,
                         static_cast<int32_t*>(c->ws[S_GOUT3].p), ws_ptr<int32_t>(c, S_STATUS),
                         c->stream);
  }));
  std::vector<int32_t> o3(3 * (size_t)A);
  CK(cudaMemcpyAsync(o3.data(), c->ws[S_GOUT3].p, sizeof(int32_t) * 3 * A, cudaMemcpyDeviceToHost,
                     c->stream));
  int32_t st = 0;
  if (slm_status s = read_status(c, &st)) return s;
  if (st) return fail(c, SLM_ECUDA, "partition disagrees with the scored split");

  // 4. next level: children of split nodes, scattered stably
  std::vector<LevelNode> next;
  std::vector<int32_t> dst(2 * (size_t)A, -1);
  int32_t pos = 0, n_split = 0;
  for (int a = 0; a < A; ++a) {
    if (!o3[3 * a]) continue;
    const LevelNode& ln = f->level[smap[a]];
    const int tree = ln.slot / f->H, h = ln.slot % f->H;
    const int32_t nl = o3[3 * a + 1], nr = o3[3 * a + 2];
    // children start on 16-byte boundaries (whole tensor-core tiles in BF16 mode)
    const int32_t pr_ = (int32_t)round_up(pos + nl, f->align);
    dst[2 * a] = pos;
    dst[2 * a + 1] = pr_;
    next.push_back(LevelNode{pos, nl, tree * f->H + 2 * h + 1, ln.depth + 1});
    next.push_back(LevelNode{pr_, nr, tree * f->H + 2 * h + 2, ln.depth + 1});
    pos = (int32_t)round_up(pr_ + nr, f->align);
    ++n_split;
  }
  if (n_split) {
    const int nx = 1 - cu;
    LevelArrays la{static_cast<float*>(f->lX[nx].p),
                   mse ? nullptr : static_cast<int32_t*>(f->lab[nx].p),
                   mse ? static_cast<float*>(f->ly[nx].p) : nullptr,
                   f->weighted ? static_cast<uint32_t*>(f->lw[nx].p) : nullptr,
                   static_cast<int32_t*>(f->lidx[nx].p)};
    CK(cudaMemcpyAsync(c->ws[S_GDST].p, dst.data(), sizeof(int32_t) * 2 * A, cudaMemcpyHostToDevice,
                       c->stream));
    CK(launch(c, SLM_K_COMPACT, 0.0, [&] {
      return launch_scatter(pr, dst_tiles, n_st, static_cast<uint8_t*>(f->side.p),
                            static_cast<int32_t*>(c->ws[S_GDST].p),
                            static_cast<int32_t*>(c->ws[S_GTILEBASE].p),
                            static_cast<int32_t*>(c->ws[S_GSTILE0].p),
                            static_cast<int32_t*>(f->lidx[cu].p), la, c->stream);
    }));
    f->cur = nx;
  }
  CK(cudaStreamSynchronize(c->stream));
  f->level.swap(next);
  ++f->depth;
  if (f->level.empty()) f->done = true;
  if (n_split_out) *n_split_out = n_split;
  return SLM_OK;
}

slm_status slm_train_tree(slm_ctx* c, const slm_params* p, const float* X, int64_t n,
                          int32_t d, const int32_t* labels, const float* y,
                          slm_forest** out) {
  slm_forest* f = nullptr;
  slm_status s = slm_forest_begin(c, p, X, n, d, labels, y, &f);
  if (s) return s;
  for (int level = 0; level <= p->max_depth + 1 && !f->done; ++level) {
    if ((s = slm_grow_level(c, f, nullptr))) {
      slm_forest_free(f);
      return s;
    }
  }
  *out = f;
  return SLM_OK;
}

slm_status slm_forest_info(const slm_forest* f, int32_t* n_trees, int32_t* heap_size,
                           int32_t* d, int64_t* evaluations) {
  if (!f) return SLM_EINVAL;
  if (n_trees) *n_trees = f->n_trees;
  if (heap_size) *heap_size = f->H;
  if (d) *d = f->d;
  if (evaluations) *evaluations = f->evaluations;
  return SLM_OK;
}

slm_status slm_forest_export(slm_ctx* c, const slm_forest* f, int32_t tree,
                             int32_t* kind, float* dir, float* zmin, float* inv_w,
                             int32_t* bin, int32_t* leaf_class, double* leaf_value,
                             int64_t* weight, double* loss, int64_t* n_left,
                             int64_t* n_right) {
  if (!c || !f || tree < 0 || tree >= f->n_trees)
    return fail(c, SLM_EINVAL, "bad forest or tree index");
  CK(cudaSetDevice(c->device));
  const size_t o = (size_t)tree * f->H, H = f->H;
  slm_status s;
  if ((s = copy_out(c, kind, f->tr.kind + o, H))) return s;
  if ((s = copy_out(c, dir, f->tr.dir + o * f->d, H * f->d))) return s;
  if ((s = copy_out(c, zmin, f->tr.zmin + o, H))) return s;
  if ((s = copy_out(c, inv_w, f->tr.inv_w + o, H))) return s;
  if ((s = copy_out(c, bin, f->tr.bin + o, H))) return s;
  if ((s = copy_out(c, leaf_class, f->tr.leaf_class + o, H))) return s;
  if ((s = copy_out(c, leaf_value, f->tr.leaf_value + o, H))) return s;
  if ((s = copy_out(c, weight, f->tr.weight + o, H))) return s;
  if ((s = copy_out(c, loss, f->tr.loss + o, H))) return s;
  if ((s = copy_out(c, n_left, f->tr.n_left + o, H))) return s;
  if ((s = copy_out(c, n_right, f->tr.n_right + o, H))) return s;
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

slm_status slm_predict(slm_ctx* c, const slm_forest* f, const float* X, int64_t n,
                       int32_t d, int32_t* class_out, double* value_out,
                       int32_t* leaf_out) {
  if (!c || !f || !X || n < 0 || d != f->d)
    return fail(c, SLM_EINVAL, "bad arguments to slm_predict");
  if (n == 0) return SLM_OK;
  CK(cudaSetDevice(c->device));
  const float* dX;
  slm_status s;
  if ((s = stage_in(c, X, (size_t)n * d, c->ws[W_X], &dX))) return s;
  // outputs: device pointers directly, host pointers through staging
  int32_t* dc = class_out;
  double* dv = value_out;
  int32_t* dl = leaf_out;
  const bool hc = class_out && !is_device_ptr(class_out);
  const bool hv = value_out && !is_device_ptr(value_out);
  const bool hl = leaf_out && !is_device_ptr(leaf_out);
  size_t off_v = ((hc ? 4 * (size_t)n : 0) + 15) & ~size_t(15);
  size_t off_l = (off_v + (hv ? 8 * (size_t)n : 0) + 15) & ~size_t(15);
  size_t total = off_l + (hl ? 4 * (size_t)n * f->n_trees : 0);
  CK(ensure(c->ws[S_OUT], total));
  unsigned char* base = static_cast<unsigned char*>(c->ws[S_OUT].p);
  if (hc) dc = reinterpret_cast<int32_t*>(base);
  if (hv) dv = reinterpret_cast<double*>(base + off_v);
  if (hl) dl = reinterpret_cast<int32_t*>(base + off_l);
  CK(launch(c, SLM_K_OTHER, 0.0, [&] {
    return launch_predict(dX, n, d, f->tr, f->n_trees, f->H, f->params.n_bins, f->K,
                          f->params.criterion, dc, dv, dl, c->stream);
  }));
  if (hc) CK(cudaMemcpyAsync(class_out, dc, 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
  if (hv) CK(cudaMemcpyAsync(value_out, dv, 8 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
  if (hl)
    CK(cudaMemcpyAsync(leaf_out, dl, 4 * (size_t)n * f->n_trees, cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

// ---- SLR Boost ---------------------------------------------------------------------

struct slm_boost {
  int device = 0;
  slm_params params{};
  int d = 0;
  int K = 1;  // outputs: 1 (regression on y) or the classes (labels)
  float base = 0.0f;
  float eta = 0.0f;
  std::vector<slm_forest*> trees;  // round-major: tree (m, k) at m * K + k
  // classification: each round's K trees grown as one forest, which owns
  // their arrays; `trees` then holds views of its trees
  std::vector<slm_forest*> rounds;
};

}  // extern "C"

namespace {

// A finished tree keeps only its arrays: the level state of its growth goes.
void release_level_state(slm_forest* f) {
  DevBuf* bufs[] = {&f->own_X, &f->side, &f->lXb};
  for (DevBuf* b : bufs) release(*b);
  for (int i = 0; i < 2; ++i) {
    release(f->lX[i]);
    release(f->lab[i]);
    release(f->ly[i]);
    release(f->lw[i]);
    release(f->lidx[i]);
  }
  f->X = nullptr;
  f->level.clear();
}

// Tree t of a finished forest as a one-tree forest that owns nothing: its
// arrays stay the forest's (which must outlive the view).
slm_forest* tree_view(const slm_forest* f, int t) {
  slm_forest* v = new (std::nothrow) slm_forest();
  if (!v) return nullptr;
  v->ctx = f->ctx;
  v->device = f->device;
  v->params = f->params;
  v->params.n_trees = 1;
  v->n = f->n;
  v->d = f->d;
  v->H = f->H;
  v->n_trees = 1;
  v->K = f->K;
  v->align = f->align;
  v->tree_id0 = f->tree_id(t);
  const size_t o = (size_t)t * f->H;
  v->tr = TreeArrays{f->tr.kind + o,       f->tr.dir + o * f->d,  f->tr.zmin + o,
                     f->tr.inv_w + o,      f->tr.bin + o,         f->tr.leaf_class + o,
                     f->tr.leaf_value + o, f->tr.weight + o,      f->tr.loss + o,
                     f->tr.n_left + o,     f->tr.n_right + o};
  v->done = true;
  v->evaluations = f->tree_evals[(size_t)t];
  v->tree_evals.assign(1, v->evaluations);
  return v;
}

// Device buffers of one boosting call, released on every exit.
struct BoostWork {
  DevBuf X, y, lab, F, r, v, loss, base;
  ~BoostWork() {
    for (DevBuf* b : {&X, &y, &lab, &F, &r, &v, &loss, &base}) release(*b);
  }
};

template <typename T>
slm_status own_copy(slm_ctx* c, const T* src, size_t count, DevBuf& buf, const T** out) {
  if (is_device_ptr(src)) {
    *out = src;
    return SLM_OK;
  }
  CK(ensure(buf, sizeof(T) * count));
  CK(cudaMemcpyAsync(buf.p, src, sizeof(T) * count, cudaMemcpyHostToDevice, c->stream));
  *out = static_cast<const T*>(buf.p);
  return SLM_OK;
}

}  // namespace

extern "C" {

slm_status slm_train_boost(slm_ctx* c, const slm_params* p, const float* X, int64_t n,
                           int32_t d, const int32_t* labels, const float* y, int32_t n_rounds,
                           float learning_rate, double* train_loss_out, slm_boost** out) {
  if (!c || !p || !X || !out || n < 1 || d < 1 || n_rounds < 0 || (!labels == !y))
    return fail(c, SLM_EINVAL, "bad arguments to slm_train_boost (exactly one of labels, y)");
  *out = nullptr;
  if (p->criterion != SLM_MSE)
    return fail(c, SLM_EINVAL, "boosting trees fit residuals: criterion SLM_MSE");
  const int K = labels ? p->n_classes : 1;
  if (labels && (K < 2 || K > kMaxClasses))
    return fail(c, SLM_EINVAL, "classification boosting needs 2 <= n_classes <= 32");
  if (!(learning_rate > 0.0f && learning_rate <= 1.0f))
    return fail(c, SLM_EINVAL, "learning_rate must be in (0, 1]");
  if (p->n_trees != 1 || p->bootstrap)
    return fail(c, SLM_EUNSUPPORTED, "boosting grows one tree per round, without bootstrap");
  CK(cudaSetDevice(c->device));
  BoostWork w;
  const float* dX;
  const float* dy = nullptr;
  const int32_t* dl = nullptr;
  if (slm_status s = own_copy(c, X, (size_t)n * d, w.X, &dX)) return s;
  if (y) {
    if (slm_status s = own_copy(c, y, (size_t)n, w.y, &dy)) return s;
  } else {
    if (slm_status s = own_copy(c, labels, (size_t)n, w.lab, &dl)) return s;
    if (slm_status s = validate_inputs(c, dl, n, K, nullptr, 0)) return s;
  }
  CK(ensure(w.F, sizeof(float) * (size_t)n * K));
  CK(ensure(w.r, sizeof(float) * (size_t)n * K));
  CK(ensure(w.v, sizeof(double) * (size_t)n));
  CK(ensure(w.loss, sizeof(double) * (size_t)(n_rounds > 0 ? n_rounds : 1)));
  CK(ensure(w.base, sizeof(float)));
  float* F = static_cast<float*>(w.F.p);
  float* r = static_cast<float*>(w.r.p);
  double* v = static_cast<double*>(w.v.p);
  double* loss = static_cast<double*>(w.loss.p);
  if (y)
    CK(launch(c, SLM_K_OTHER, 0.0, [&] {
      return launch_boost_init(dy, n, F, static_cast<float*>(w.base.p), c->stream);
    }));
  else
    CK(launch(c, SLM_K_OTHER, 0.0,
              [&] { return launch_fill_f(F, 0.0f, n * K, c->stream); }));
  std::unique_ptr<slm_boost, void (*)(slm_boost*)> b(new (std::nothrow) slm_boost,
                                                     slm_boost_free);
  if (!b) return fail(c, SLM_ENOMEM, "boost handle");
  b->device = c->device;
  b->params = *p;
  b->params.n_classes = 0;
  b->d = d;
  b->K = K;
  b->eta = learning_rate;
  for (int32_t m = 1; m <= n_rounds; ++m) {
    // residuals of every output from the same F
    if (y)
      CK(launch(c, SLM_K_OTHER, 0.0,
                [&] { return launch_boost_residual(dy, F, r, n, c->stream); }));
    else
      CK(launch(c, SLM_K_OTHER, 0.0,
                [&] { return launch_softmax_residual(F, dl, n, K, r, c->stream); }));
    // the round's trees: one tree on y (regression), or the K class trees
    // grown together as one forest (tree k fits class k's residuals, global
    // tree id k, the round's key seed + m), every level of all K searched in
    // one batch
    slm_forest* round = nullptr;
    if (K > 1) {
      slm_params q = b->params;
      q.seed = p->seed + (uint64_t)m;
      q.n_trees = K;
      if (slm_status s = forest_begin_impl(c, &q, dX, n, d, nullptr, r, true, 0, 1, &round))
        return s;
      b->rounds.push_back(round);
      for (int level = 0; level <= q.max_depth + 1 && !round->done; ++level)
        if (slm_status s = slm_grow_level(c, round, nullptr)) return s;
      release_level_state(round);
    }
    for (int k = 0; k < K; ++k) {
      slm_params q = b->params;
      q.seed = p->seed + (uint64_t)m;
      slm_forest* f = nullptr;
      if (round) {
        f = tree_view(round, k);
        if (!f) return fail(c, SLM_ENOMEM, "host allocation failed");
      } else if (slm_status s = slm_train_tree(c, &q, dX, n, d, nullptr, r, &f)) {
        return s;
      }
      b->trees.push_back(f);
      if (!round) release_level_state(f);
      CK(launch(c, SLM_K_OTHER, 0.0, [&] {
        return launch_predict(dX, n, d, f->tr, 1, f->H, q.n_bins, 1, SLM_MSE, nullptr, v,
                              nullptr, c->stream);
      }));
      CK(launch(c, SLM_K_OTHER, 0.0, [&] {
        return launch_boost_update(F, v, learning_rate, n, c->stream, K, k);
      }));
    }
    if (y)
      CK(launch(c, SLM_K_OTHER, 0.0,
                [&] { return launch_boost_mse(dy, F, n, loss + (m - 1), c->stream); }));
    else
      CK(launch(c, SLM_K_OTHER, 0.0,
                [&] { return launch_boost_ce(F, dl, n, K, loss + (m - 1), c->stream); }));
  }
  if (y)
    CK(cudaMemcpyAsync(&b->base, w.base.p, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  if (train_loss_out && n_rounds > 0)
    CK(cudaMemcpyAsync(train_loss_out, loss, sizeof(double) * n_rounds, cudaMemcpyDefault,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (slm_status s = check_kernel_errors(c)) return s;
  *out = b.release();
  return SLM_OK;
}

slm_status slm_boost_predict(slm_ctx* c, const slm_boost* b, const float* X, int64_t n,
                             int32_t d, float* value_out, int32_t* class_out) {
  if (!c || !b || !X || (!value_out && !class_out) || n < 0 || d != b->d ||
      (class_out && b->K < 2))
    return fail(c, SLM_EINVAL, "bad arguments to slm_boost_predict");
  if (n == 0) return SLM_OK;
  CK(cudaSetDevice(c->device));
  const float* dX;
  if (slm_status s = stage_in(c, X, (size_t)n * d, c->ws[W_X], &dX)) return s;
  const int K = b->K;
  const size_t off_f = (sizeof(double) * (size_t)n + 15) & ~size_t(15);
  const size_t off_c = (off_f + sizeof(float) * (size_t)n * K + 15) & ~size_t(15);
  CK(ensure(c->ws[S_OUT], off_c + sizeof(int32_t) * (size_t)n));
  unsigned char* base = static_cast<unsigned char*>(c->ws[S_OUT].p);
  double* v = reinterpret_cast<double*>(base);
  float* F = value_out && is_device_ptr(value_out) ? value_out
                                                   : reinterpret_cast<float*>(base + off_f);
  int32_t* cls = class_out && is_device_ptr(class_out)
                     ? class_out
                     : reinterpret_cast<int32_t*>(base + off_c);
  CK(launch(c, SLM_K_OTHER, 0.0,
            [&] { return launch_fill_f(F, K == 1 ? b->base : 0.0f, n * K, c->stream); }));
  for (size_t t = 0; t < b->trees.size(); ++t) {
    const slm_forest* f = b->trees[t];
    CK(launch(c, SLM_K_OTHER, 0.0, [&] {
      return launch_predict(dX, n, d, f->tr, 1, f->H, b->params.n_bins, 1, SLM_MSE, nullptr,
                            v, nullptr, c->stream);
    }));
    CK(launch(c, SLM_K_OTHER, 0.0, [&] {
      return launch_boost_update(F, v, b->eta, n, c->stream, K, (int)(t % K));
    }));
  }
  if (class_out)
    CK(launch(c, SLM_K_OTHER, 0.0, [&] { return launch_argmax_rows(F, n, K, cls, c->stream); }));
  if (value_out && F != value_out)
    CK(cudaMemcpyAsync(value_out, F, sizeof(float) * (size_t)n * K, cudaMemcpyDeviceToHost,
                       c->stream));
  if (class_out && cls != class_out)
    CK(cudaMemcpyAsync(class_out, cls, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

slm_status slm_boost_info(const slm_boost* b, int32_t* n_rounds, int32_t* n_outputs,
                          float* base, float* learning_rate) {
  if (!b) return SLM_EINVAL;
  if (n_rounds) *n_rounds = (int32_t)(b->trees.size() / b->K);
  if (n_outputs) *n_outputs = b->K;
  if (base) *base = b->base;
  if (learning_rate) *learning_rate = b->eta;
  return SLM_OK;
}

const slm_forest* slm_boost_tree(const slm_boost* b, int32_t m) {
  if (!b || m < 0 || m >= (int32_t)b->trees.size()) return nullptr;
  return b->trees[m];
}

void slm_boost_free(slm_boost* b) {
  if (!b) return;
  for (slm_forest* f : b->trees) slm_forest_free(f);  // (views first)
  for (slm_forest* f : b->rounds) slm_forest_free(f);
  delete b;
}

// ---- learned swarm proposal ------------------------------------------------------

namespace {
constexpr size_t kNW1 = (size_t)kPropIn * kPropH, kNW2 = (size_t)kPropH * kPropH,
                 kNW3 = (size_t)kPropH * kPropOut;
constexpr size_t kNParams = kNW1 + kPropH + kNW2 + kPropH + kNW3 + kPropOut;

// Views of a parameter-sized block: W1, b1, W2, b2, W3, b3 in this order.
void split_params(float* b, float** W1, float** b1, float** W2, float** b2, float** W3,
                  float** b3) {
  *W1 = b;
  *b1 = *W1 + kNW1;
  *W2 = *b1 + kPropH;
  *b2 = *W2 + kNW2;
  *W3 = *b2 + kPropH;
  *b3 = *W3 + kNW3;
}
}  // namespace

slm_status slm_proposal_create(slm_ctx* c, uint64_t seed, slm_proposal** out) {
  if (!c || !out) return SLM_EINVAL;
  *out = nullptr;
  CK(cudaSetDevice(c->device));
  slm_proposal* pp = new (std::nothrow) slm_proposal();
  if (!pp) return fail(c, SLM_ENOMEM, "host allocation failed");
  pp->device = c->device;
  // params | grads | Adam m | Adam v (FP32), then the bfloat16 weight copies
  const size_t bytes = sizeof(float) * 4 * kNParams + 2 * (kNW1 + kNW2 + kNW3) + 256;
  cudaError_t e = ensure(pp->mem, bytes);
  if (e) {
    delete pp;
    return cuda_fail(c, e, "proposal memory");
  }
  float* base = static_cast<float*>(pp->mem.p);
  MlpParams& m = pp->m;
  split_params(base, &m.W1, &m.b1, &m.W2, &m.b2, &m.W3, &m.b3);
  MlpGrads& g = pp->g;
  split_params(base + kNParams, &g.W1, &g.b1, &g.W2, &g.b2, &g.W3, &g.b3);
  MlpState& st = pp->s;
  split_params(base + 2 * kNParams, &st.mW1, &st.mb1, &st.mW2, &st.mb2, &st.mW3, &st.mb3);
  split_params(base + 3 * kNParams, &st.vW1, &st.vb1, &st.vW2, &st.vb2, &st.vW3, &st.vb3);
  __nv_bfloat16* bb = reinterpret_cast<__nv_bfloat16*>(base + 4 * kNParams);
  m.W1b = bb;
  m.W2b = bb + kNW1;
  m.W3b = bb + kNW1 + kNW2;
  if ((e = cudaMemsetAsync(base + 2 * kNParams, 0, sizeof(float) * 2 * kNParams, c->stream)) ||
      (e = launch_mlp_init(m, seed, c->stream)) || (e = cudaStreamSynchronize(c->stream))) {
    release(pp->mem);
    delete pp;
    return cuda_fail(c, e, "proposal init");
  }
  c->launches += 7;
  *out = pp;
  return SLM_OK;
}

void slm_proposal_free(slm_proposal* pp) {
  if (!pp) return;
  cudaSetDevice(pp->device);
  release(pp->mem);
  delete pp;
}

slm_status slm_proposal_set(slm_ctx* c, slm_proposal* pp, const float* W1, const float* b1,
                            const float* W2, const float* b2, const float* W3, const float* b3) {
  if (!c || !pp || !W1 || !b1 || !W2 || !b2 || !W3 || !b3)
    return fail(c, SLM_EINVAL, "NULL argument");
  CK(cudaSetDevice(c->device));
  const float* src[6] = {W1, b1, W2, b2, W3, b3};
  float* dst[6] = {pp->m.W1, pp->m.b1, pp->m.W2, pp->m.b2, pp->m.W3, pp->m.b3};
  const size_t cnt[6] = {kNW1, kPropH, kNW2, kPropH, kNW3, kPropOut};
  for (int i = 0; i < 6; ++i)
    CK(cudaMemcpyAsync(dst[i], src[i], sizeof(float) * cnt[i], cudaMemcpyDefault, c->stream));
  CK(cudaMemsetAsync(pp->s.mW1, 0, sizeof(float) * 2 * kNParams, c->stream));
  CK(launch(c, SLM_K_PROPOSAL, 0.0, [&] { return launch_mlp_sync_bf16(pp->m, c->stream); }));
  pp->step = 0;
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

slm_status slm_proposal_get(slm_ctx* c, const slm_proposal* pp, float* W1, float* b1, float* W2,
                            float* b2, float* W3, float* b3) {
  if (!c || !pp) return fail(c, SLM_EINVAL, "NULL argument");
  CK(cudaSetDevice(c->device));
  float* dst[6] = {W1, b1, W2, b2, W3, b3};
  const float* src[6] = {pp->m.W1, pp->m.b1, pp->m.W2, pp->m.b2, pp->m.W3, pp->m.b3};
  const size_t cnt[6] = {kNW1, kPropH, kNW2, kPropH, kNW3, kPropOut};
  for (int i = 0; i < 6; ++i)
    if (dst[i])
      CK(cudaMemcpyAsync(dst[i], src[i], sizeof(float) * cnt[i], cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

slm_status slm_proposal_forward(slm_ctx* c, const slm_proposal* pp, const float* stats,
                                int32_t n, float* out) {
  if (!c || !pp || !stats || !out || n < 1) return fail(c, SLM_EINVAL, "bad arguments");
  CK(cudaSetDevice(c->device));
  const float* ds;
  if (slm_status s = stage_in(c, stats, (size_t)n * kPropIn, c->ws[W_PS], &ds)) return s;
  MlpWork w;
  if (slm_status s = proposal_work(c, n, &w)) return s;
  CK(launch(c, SLM_K_PROPOSAL, 0.0, [&] { return launch_mlp_forward(pp->m, ds, n, w, c->stream); }));
  CK(cudaMemcpyAsync(out, w.O, sizeof(float) * (size_t)n * kPropOut, cudaMemcpyDefault,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

namespace {
slm_status check_train_args(slm_ctx* c, const float* stats, const int32_t* dims,
                            const float* targets, int32_t n) {
  if (!stats || !dims || !targets || n < 1) return fail(c, SLM_EINVAL, "bad arguments");
  std::vector<int32_t> hd((size_t)n);
  CK(cudaMemcpy(hd.data(), dims, sizeof(int32_t) * (size_t)n, cudaMemcpyDefault));
  for (int32_t v : hd)
    if (v < 1 || v > kPropD) return fail(c, SLM_EINVAL, "dims must be in [1, 256]");
  return SLM_OK;
}
}  // namespace

slm_status slm_proposal_loss_grad(slm_ctx* c, const slm_proposal* pp, const float* stats,
                                  const int32_t* dims, const float* targets, int32_t n,
                                  double* loss, float* gW1, float* gb1, float* gW2, float* gb2,
                                  float* gW3, float* gb3) {
  if (!c || !pp) return SLM_EINVAL;
  CK(cudaSetDevice(c->device));
  if (slm_status s = check_train_args(c, stats, dims, targets, n)) return s;
  const float *ds, *dt;
  const int32_t* dd;
  slm_status s;
  if ((s = stage_in(c, stats, (size_t)n * kPropIn, c->ws[W_PS], &ds)) ||
      (s = stage_in(c, dims, (size_t)n, c->ws[W_PD], &dd)) ||
      (s = stage_in(c, targets, (size_t)n * kPropD, c->ws[W_PT], &dt)))
    return s;
  MlpWork w;
  if ((s = proposal_work(c, n, &w))) return s;
  CK(ensure(c->ws[S_PLOSS], 2 * sizeof(double)));
  double* dl = ws_ptr<double>(c, S_PLOSS);
  CK(launch(c, SLM_K_PROPOSAL, 0.0, [&] {
    return launch_mlp_loss_grad(pp->m, ds, dd, dt, n, w, pp->g, dl, c->stream);
  }));
  if (loss) CK(cudaMemcpyAsync(loss, dl, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  float* dst[6] = {gW1, gb1, gW2, gb2, gW3, gb3};
  const float* src[6] = {pp->g.W1, pp->g.b1, pp->g.W2, pp->g.b2, pp->g.W3, pp->g.b3};
  const size_t cnt[6] = {kNW1, kPropH, kNW2, kPropH, kNW3, kPropOut};
  for (int i = 0; i < 6; ++i)
    if (dst[i])
      CK(cudaMemcpyAsync(dst[i], src[i], sizeof(float) * cnt[i], cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

slm_status slm_proposal_train(slm_ctx* c, slm_proposal* pp, const float* stats,
                              const int32_t* dims, const float* targets, int32_t n,
                              int32_t epochs, int32_t batch, float lr, uint64_t seed,
                              double* epoch_loss) {
  if (!c || !pp) return SLM_EINVAL;
  if (epochs < 0 || batch < 1 || !(lr > 0.0f) || !std::isfinite(lr))
    return fail(c, SLM_EINVAL, "bad epochs / batch / lr");
  CK(cudaSetDevice(c->device));
  if (slm_status s = check_train_args(c, stats, dims, targets, n)) return s;
  const float *ds, *dt;
  const int32_t* dd;
  slm_status s;
  if ((s = stage_in(c, stats, (size_t)n * kPropIn, c->ws[W_PS], &ds)) ||
      (s = stage_in(c, dims, (size_t)n, c->ws[W_PD], &dd)) ||
      (s = stage_in(c, targets, (size_t)n * kPropD, c->ws[W_PT], &dt)))
    return s;
  const int b = std::min(batch, n);
  MlpWork w;
  if ((s = proposal_work(c, b, &w))) return s;
  CK(ensure(c->ws[W_PIDX], sizeof(int32_t) * (size_t)n));
  CK(ensure(c->ws[W_PBS], sizeof(float) * (size_t)b * kPropIn));
  CK(ensure(c->ws[W_PBD], sizeof(int32_t) * (size_t)b));
  CK(ensure(c->ws[W_PBT], sizeof(float) * (size_t)b * kPropD));
  CK(ensure(c->ws[S_PLOSS], 2 * sizeof(double)));
  double* dl = ws_ptr<double>(c, S_PLOSS);
  int32_t* didx = ws_ptr<int32_t>(c, W_PIDX);
  float* bs = ws_ptr<float>(c, W_PBS);
  int32_t* bd = ws_ptr<int32_t>(c, W_PBD);
  float* bt = ws_ptr<float>(c, W_PBT);
  std::vector<int32_t> order((size_t)n);
  std::mt19937_64 rng(seed);
  for (int32_t ep = 0; ep < epochs; ++ep) {
    std::iota(order.begin(), order.end(), 0);
    std::shuffle(order.begin(), order.end(), rng);
    CK(cudaMemcpyAsync(didx, order.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemsetAsync(dl + 1, 0, sizeof(double), c->stream));
    int nb = 0;
    for (int32_t r0 = 0; r0 < n; r0 += b, ++nb) {
      const int bn = std::min(b, n - r0);
      CK(launch(c, SLM_K_PROPOSAL, 0.0, [&] {
        cudaError_t e;
        if ((e = launch_gather_rows(ds, kPropIn, didx + r0, bn, bs, c->stream)) ||
            (e = launch_gather_rows(dd, 1, didx + r0, bn, bd, c->stream)) ||
            (e = launch_gather_rows(dt, kPropD, didx + r0, bn, bt, c->stream)))
          return e;
        if ((e = launch_mlp_loss_grad(pp->m, bs, bd, bt, bn, w, pp->g, dl, c->stream))) return e;
        if ((e = launch_adam(pp->m, pp->s, pp->g, (int)++pp->step, lr, c->stream))) return e;
        return launch_acc_double(dl + 1, dl, c->stream);
      }));
    }
    double tot = 0.0;
    CK(cudaMemcpyAsync(&tot, dl + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    // the order vector is reused by the next epoch's copy: wait for this one
    CK(cudaStreamSynchronize(c->stream));
    if (epoch_loss) epoch_loss[ep] = tot / nb;
  }
  return SLM_OK;
}

slm_status slm_use_proposal(slm_ctx* c, const slm_proposal* pp) {
  if (!c) return SLM_EINVAL;
  if (pp && pp->device != c->device) return fail(c, SLM_EINVAL, "proposal on another device");
  c->prop = pp;
  return SLM_OK;
}

slm_status slm_swarm_seed(slm_ctx* c, uint64_t seed, uint32_t node_uid, int32_t P, int32_t d,
                          const float* mu_hat, const float* rho, float* pos) {
  if (!c || !mu_hat || !rho || !pos || P < 1 || d < 1 || d > kMaxD)
    return fail(c, SLM_EINVAL, "bad arguments");
  CK(cudaSetDevice(c->device));
  const float *dm, *dr;
  slm_status s;
  if ((s = stage_in(c, mu_hat, (size_t)d, c->ws[W_PMU], &dm)) ||
      (s = stage_in(c, rho, (size_t)P, c->ws[W_PRHO], &dr)))
    return s;
  float* dp = pos;
  const bool dev = is_device_ptr(pos);
  if (!dev) {
    CK(ensure(c->ws[W_PPOS], sizeof(float) * (size_t)P * d));
    dp = ws_ptr<float>(c, W_PPOS);
  }
  CK(launch(c, SLM_K_PROPOSAL, 0.0, [&] {
    return launch_seed_positions(seed, node_uid, P, d, dm, dr, dp, c->stream);
  }));
  if (!dev)
    CK(cudaMemcpyAsync(pos, dp, sizeof(float) * (size_t)P * d, cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

slm_status slm_node_stats(slm_ctx* c, const float* X, int64_t n, int32_t d,
                          const int32_t* labels, int32_t n_classes, const float* y,
                          const int32_t* sample_idx, const uint32_t* weights, int64_t n_idx,
                          float* stats) {
  if (!c || !stats) return SLM_EINVAL;
  slm_params p{};
  p.criterion = labels ? SLM_GINI : SLM_MSE;
  p.n_classes = labels ? n_classes : 0;
  p.n_bins = 2;
  p.min_leaf = 1;
  if (d > kPropD || (labels && n_classes > kPropK))
    return fail(c, SLM_EUNSUPPORTED, "node statistics need d <= 256 and n_classes <= 20");
  if (slm_status s = check_node_args(c, &p, X, n, d, labels, y, sample_idx, &n_idx, false))
    return s;
  CK(cudaSetDevice(c->device));
  Problem pr;
  if (slm_status s = prepare_node(c, &p, X, n, d, labels, y, sample_idx, weights, n_idx, 1, &pr))
    return s;
  const std::vector<NodeDesc> nodes{NodeDesc{0, (int32_t)n_idx, 0u, -1}};
  CK(ensure(c->ws[S_NODES], sizeof(NodeDesc)));
  CK(cudaMemcpyAsync(c->ws[S_NODES].p, nodes.data(), sizeof(NodeDesc), cudaMemcpyHostToDevice,
                     c->stream));
  float* ds = nullptr;
  if (slm_status s = batch_stats(c, pr, nodes, &ds)) return s;
  CK(cudaMemcpyAsync(stats, ds, sizeof(float) * kPropIn, cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SLM_OK;
}

slm_status slm_profile(slm_ctx* c, int on) {
  if (!c) return SLM_EINVAL;
  CK(cudaSetDevice(c->device));
  CK(collect_profile(c));
  c->prof = on != 0;
  for (int k = 0; k < SLM_K_COUNT; ++k) {
    c->k_launches[k] = 0;
    c->k_ms[k] = 0.0;
    c->k_pairs[k] = 0.0;
  }
  return SLM_OK;
}

slm_status slm_kernel_stats(slm_ctx* c, int32_t kernel, int64_t* launches,
                            double* total_ms, double* pairs) {
  if (!c || kernel < 0 || kernel >= SLM_K_COUNT) return fail(c, SLM_EINVAL, "bad kernel id");
  CK(cudaSetDevice(c->device));
  CK(collect_profile(c));
  if (launches) *launches = c->k_launches[kernel];
  if (total_ms) *total_ms = c->k_ms[kernel];
  if (pairs) *pairs = c->k_pairs[kernel];
  return SLM_OK;
}

slm_status slm_launch_count(slm_ctx* c, int64_t* launches) {
  if (!c || !launches) return SLM_EINVAL;
  *launches = c->launches;
  return SLM_OK;
}

slm_status slm_set_fused_step(slm_ctx* c, int32_t on, int64_t* searches) {
  if (!c) return SLM_EINVAL;
  if (on < 0 || on > 2) return fail(c, SLM_EINVAL, "on must be 0, 1 or 2");
  c->fused_step = on;
  if (searches) *searches = c->fused_searches;
  return SLM_OK;
}

slm_status slm_set_step_shape(slm_ctx* c, int32_t shape, int32_t* last) {
  if (!c) return SLM_EINVAL;
  if (shape < -1 || shape >= kStepShapeCount)
    return fail(c, SLM_EINVAL, "shape must be -1 or 0 .. 5");
  c->step_shape = shape;
  if (last) *last = c->last_step_shape;
  return SLM_OK;
}

slm_status slm_set_tree_ids(slm_ctx* c, int64_t first, int64_t stride) {
  if (!c || first < 0 || stride < 1 || first > 65535 || stride > 65535) return SLM_EINVAL;
  c->tree_id0 = first;
  c->tree_stride = stride;
  return SLM_OK;
}

slm_status slm_set_class_hist(slm_ctx* c, int32_t on, int32_t node_step) {
  if (!c) return SLM_EINVAL;
  c->class_hist = on != 0;
  c->node_step = node_step != 0;
  return SLM_OK;
}

slm_status slm_set_projection_tma(slm_ctx* c, int32_t on) {
  if (!c) return SLM_EINVAL;
  c->tma = on != 0;
  return SLM_OK;
}

slm_status slm_test_hooks(slm_ctx* c, int32_t first_wait_polls, int64_t fail_alloc_after) {
  if (!c || fail_alloc_after < 0) return fail(c, SLM_EINVAL, "bad test hook values");
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(c->stream));
  CK(set_first_wait_polls(first_wait_polls));
  g_fail_alloc.store(fail_alloc_after);
  return SLM_OK;
}

slm_status slm_set_node_search(slm_ctx* c, int32_t on) {
  if (!c || (on != 0 && on != 1)) return fail(c, SLM_EINVAL, "node search must be 0 or 1");
  c->node_search = on == 1;
  return SLM_OK;
}

slm_status slm_last_node_search(slm_ctx* c, int32_t* ctas_per_node) {
  if (!c || !ctas_per_node) return SLM_EINVAL;
  *ctas_per_node = c->last_node_search;
  return SLM_OK;
}

slm_status slm_set_small_nodes(slm_ctx* c, int32_t max_entries, int64_t min_pairs) {
  if (!c || max_entries < 0 || min_pairs < -1)
    return fail(c, SLM_EINVAL, "small nodes: max_entries >= 0, min_pairs >= -1");
  c->small_node_max = max_entries;
  c->small_min_pairs = min_pairs;
  return SLM_OK;
}

slm_status slm_set_tuning(slm_ctx* c, int32_t on) {
  if (!c || (on != 0 && on != 1)) return fail(c, SLM_EINVAL, "tuning must be 0 or 1");
  c->tune = on;
  return SLM_OK;
}

slm_status slm_force_tiles(slm_ctx* c, int32_t pg, int32_t ctas_per_sm, int32_t gather) {
  if (!c) return SLM_EINVAL;
  if (pg == 0) {
    c->forced = slm_ctx::Tiles{0, 0};
    return SLM_OK;
  }
  if ((pg != 8 && pg != 16 && pg != 24 && pg != 32 && pg != 48) ||
      (ctas_per_sm != 1 && ctas_per_sm != 2) || (gather != 0 && gather != 1))
    return fail(c, SLM_EINVAL,
                "tiles: particles per group 8/16/24/32/48, 1 or 2 CTAs per SM, gather 0/1");
  c->forced = slm_ctx::Tiles{pg, ctas_per_sm, 0.f, gather == 1};
  return SLM_OK;
}

slm_status slm_tuning_stats(slm_ctx* c, int64_t* shapes, int32_t* last_pg,
                            int32_t* last_ctas_per_sm, int32_t* last_hist_cluster) {
  if (!c) return SLM_EINVAL;
  if (shapes) *shapes = (int64_t)c->tuned.size();
  if (last_pg) *last_pg = c->last.pg;
  if (last_ctas_per_sm) *last_ctas_per_sm = c->last.cps;
  if (last_hist_cluster) *last_hist_cluster = c->last_split;
  return SLM_OK;
}

slm_status slm_tuned_shapes(slm_ctx* c, int32_t max, int32_t* n, int32_t* d, int32_t* pp,
                            int32_t* tiles_log2, int32_t* pg, int32_t* ctas_per_sm,
                            int32_t* gather, float* ms) {
  if (!c || !n || max < 0) return SLM_EINVAL;
  int32_t i = 0;
  for (const auto& kv : c->tuned) {
    if (i < max) {
      if (d) d[i] = (int32_t)(kv.first >> 40);
      if (pp) pp[i] = (int32_t)((kv.first >> 16) & 0xFFFFFF);
      if (tiles_log2) tiles_log2[i] = (int32_t)(kv.first & 0x3FFF);
      if (pg) pg[i] = kv.second.pg;
      if (ctas_per_sm) ctas_per_sm[i] = kv.second.cps;
      if (gather) gather[i] = kv.second.gather ? 1 : (kv.second.tma && (kv.first >> 14 & 1)) ? 2 : 0;
      if (ms) ms[i] = kv.second.ms;
    }
    ++i;
  }
  *n = i;
  return SLM_OK;
}

slm_status slm_set_graphs(slm_ctx* c, int32_t on) {
  if (!c || (on != 0 && on != 1)) return fail(c, SLM_EINVAL, "graphs must be 0 or 1");
  c->graphs = on != 0;
  return SLM_OK;
}

slm_status slm_graph_stats(slm_ctx* c, int64_t* launches, int64_t* reuses, int64_t* updates,
                           int64_t* instantiations) {
  if (!c) return SLM_EINVAL;
  if (launches) *launches = c->graph_launches;
  if (reuses) *reuses = c->graph_reuses;
  if (updates) *updates = c->graph_updates;
  if (instantiations) *instantiations = c->graph_instantiations;
  return SLM_OK;
}

}  // extern "C"
