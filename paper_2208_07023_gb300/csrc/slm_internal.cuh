// Internal declarations of libslm: shared layouts and kernel launchers.
// Nothing here is part of the public C ABI (include/slm.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include "slm.h"

namespace slm {

// ---- compile-time tiling ----------------------------------------------------
constexpr int kThreads = 256;   // threads per CTA for the evaluation kernels
constexpr int kPG = 16;         // particles per CTA ("particle group"); Pp pads to it
constexpr int kPGMax = 48;      // widest particle group of the projection
constexpr int kTS = 256;        // samples per tile: 8 warps x 32 samples
constexpr int kKC = 32;         // features per smem chunk of the projection
constexpr int kXS = kKC + 4;    // padded smem row stride (floats): rows r and
                                // r+1 start 4 banks apart -> conflict-free
constexpr int kMaxBins = 256;
constexpr int kMaxClasses = 32;
constexpr int kMaxHistBytesPerParticle = 10240;  // B*K*4 (classification)
constexpr int kMaxParticles = 256;
constexpr int kMaxD = 1024;
constexpr int kProbMaxR = 64;  // coefficients per candidate of the probabilistic search
// bfloat16 projection on the tensor cores (SLM_PROJ_BF16_TOPK)
constexpr int kMmaRows = 128;                // rows per MMA tile = TMEM lanes
constexpr int kMmaMaxBBytes = 128 * 1024;    // staged positions: Pp * dp * 2
// learned swarm proposal: inputs padded to 256 features x (20 classes + 1)
constexpr int kPropD = 256, kPropK = 20, kPropIn = 256 * 21, kPropH = 512, kPropP = 64;
constexpr int kPropOut = kPropD + kPropP;

// Philox stream purposes (high byte of counter word 3).
enum Purpose : uint32_t {
  kInitX = 1,
  kInitV = 2,
  kR1 = 3,
  kR2 = 4,
  kBootstrap = 5,
  kApso = 7  // the adaptive PSO step size delta, counter (uid, t, 0, 0)
};

// Score of one projection on one node. Same meaning as slm_eval.
struct EvalRes {
  double loss;
  uint64_t num, den;
  float zmin, inv_w;
  int32_t bin, valid;
  int64_t nl, nr;
};
static_assert(sizeof(EvalRes) == sizeof(slm_eval), "layout");

// One node searched in a batch.
struct NodeDesc {
  int32_t seg_start;  // first entry in the level's idx / w arrays
  int32_t seg_len;    // number of entries (distinct samples)
  uint32_t uid;       // Philox node uid
  int32_t slot;       // tree * H + heap index, or -1
};

// A tile of up to kTS consecutive rows of one node (projection work unit,
// together with a particle group).
struct WorkTile {
  int32_t node;  // index into the batch's NodeDesc array
  int32_t row0;  // first entry (absolute row of the level arrays)
  int32_t rows;  // <= kTS
  int32_t pad;
};

// Problem data shared by all nodes of a batch (passed by value). Rows are
// stored entry-ordered: node a owns entries [seg_start, seg_start + seg_len).
struct Problem {
  const float* X;         // [E, d] rows of the entries
  // optional: the base rows [n, d] and each entry's row in them; the FP32
  // projection may read entry e's row as Xg[gidx[e]] instead of X[e]
  const float* Xg;
  const int32_t* gidx;
  const int32_t* lab;     // [E] labels (classification) or null
  const float* y;         // [E] targets (MSE) or null
  const uint32_t* w;      // [E] multiplicities or null (= 1)
  int64_t E;              // entries in the batch
  int64_t Ez;             // row stride of z: E rounded up to a multiple of 4
  int32_t d;
  int32_t crit;           // slm_criterion
  int32_t K;              // classes (1 for MSE)
  int32_t B;
  int32_t min_leaf;
  int32_t P;              // particles
  int32_t Pp;             // padded to a multiple of kPG
  int32_t G;              // Pp / kPG
  // SLM_PROJ_BF16_TOPK: the rows in bfloat16, in the tensor-core operand
  // layout of launch_to_mma_layout (kMmaRows-row blocks), d padded to dp
  const uint16_t* Xb;
  int32_t dp;             // d rounded up to a multiple of 16
  // MSE: per entry, w (y - c) and w (y - c)^2 in fixed point (c = the node's
  // mid-range); mscale[2a], mscale[2a+1]: value of one unit of each
  const long long* m1;
  const long long* m2;
  const double* mscale;
};

// Codes of the kernels' error word (Swarm::err). Both mean that a bounded
// wait gave up: the host reports them as SLM_ETIMEOUT; any other non-zero
// value is reported as SLM_ECUDA.
constexpr int32_t kErrCopyTimeout = 3;  // a bulk / tensor-map copy did not land
constexpr int32_t kErrMmaTimeout = 4;   // a tensor-core stage did not complete
__host__ __device__ inline bool err_is_timeout(int32_t e) {
  return e == kErrCopyTimeout || e == kErrMmaTimeout;
}

struct SwarmCoef {
  float inertia, c1, c2;
  uint64_t seed;
};

// Device swarm state of A nodes.
struct Swarm {
  float* pos;     // [A, Pp, d]
  float* vel;     // [A, Pp, d]
  float* pbest;   // [A, Pp, d]
  float* gbest;   // [A, d]
  EvalRes* cur;   // [A, Pp]   scores of the current positions
  EvalRes* pb;    // [A, Pp]   pbest scores
  EvalRes* gb;    // [2, A]    gbest score after iteration t in gb[(t & 1) * A + a]
  int32_t* gpart; // [A]
  int32_t* giter; // [A]
  double* trace;  // [A, T+1] or null
  int32_t* zmm;   // [A, Pp, 2] ordered-int range of each projection
  float* z;       // [P, E] projections of the current iteration
  int32_t* done;  // [A] particle groups of the node scored in this iteration
  int32_t* err;   // kernel error word (0, or a kErr* code)
  int32_t T;
  // SLM_PROJ_BF16_TOPK: sel[A, k] re-scored particles of each node in
  // increasing order; non-null when the gbest step runs in k_merge
  const int32_t* sel;
  int32_t k;
  // SLM_PROJ_BF16_TOPK, histogram of the reduced pass: when tk_sel is set,
  // the last CTA to score a node (counter done[a], left at 0) selects its
  // tk_k best particles into tk_sel[A, tk_k] (increasing order), tk_inv[A, Pp]
  // (rank in tk_sel or -1) and their positions into tk_pos[A, tk_kp, d]
  int32_t* tk_sel;
  int32_t* tk_inv;
  float* tk_pos;
  int32_t tk_k, tk_kp;
  // when set, the swarm kernels also write the positions as bfloat16 MMA
  // operands: posb[A, Pp * dp] (layout of launch_to_mma_layout, R = Pp)
  uint16_t* posb;
  // adaptive PSO: per node the state and the next move's inertia and
  // learning factors (null: the fixed coefficients of SwarmCoef). The
  // evaluation then scores one slot more than the swarm has particles: slot
  // P (the swarm's P) holds the elite candidate, and k_apso, not k_move,
  // takes the gbest step
  struct ApsoState* apso;
  // the move folded into the next projection (k_step): when ic is set, the
  // histogram kernels follow each particle's pbest step of evaluation t < T
  // with the terms of Eq. pso-1 that do not depend on gB, for the move to
  // t + 1 with the coefficients `co`: ic[A, Pp, d] = omega v + (c1 r1)(pB - x)
  // and s2[A, Pp, d] = c2 r2; k_step then adds (s2 (gB - x)) after the gbest
  // step. Positions alternate between two buffers by iteration parity (pos is
  // the one of the iteration being scored)
  float* ic;
  float* s2;
  SwarmCoef co;
  // with node_step set (classification searches whose nodes all go to
  // k_hist_cls): the last CTA to score a node in evaluation t (counter
  // done[a], left at 0) takes the node's gbest step (the rule of k_move)
  // and, for t < T, moves its particles into pos_next; k_step then only
  // loads positions. n_nodes: the batch's node count (stride of gb).
  float* pos_next;
  int32_t node_step;
  int32_t n_nodes;
  // folded searches: imp[(t & 1) * n_nodes + a] != 0 iff some particle of
  // node a scored strictly better than gB in evaluation t (set by the
  // histogram kernels, reset by the kernel that takes the gbest step); the
  // gbest step skips its argmin when it is 0, since gB then stays
  int32_t* imp;
};

// Adaptive PSO state of one node (Sec. III-B): evolutionary state 1..4
// (exploration, exploitation, convergence, jumping out), whether an elite
// candidate waits in slot P for the next evaluation, and the inertia and
// learning factors of the next move.
struct ApsoState {
  int32_t state;
  int32_t pending;
  float c1, c2, w;
};

// Nodes of at most this many entries are scored by the warp-per-particle
// histogram kernel in classification searches.
constexpr int kWarpNodeMax = 4096;

// The histogram kernel's first-wait polls on the current device (< 0: the
// default bound); a test hook for the timeout path.
cudaError_t set_first_wait_polls(int polls);
// c ln c is tabulated for counts below this (8 MB of doubles per device).
constexpr int kXlogxTab = 1 << 20;
// Builds the device's c ln c table once per process (synchronous).
cudaError_t ensure_xlogx_table(int device);
// The device's table (c ln c for c < kXlogxTab), null before it is built.
const double* xlogx_table(int device);

// ---- launchers (eval_kernels.cu) -------------------------------------------
cudaError_t prepare_eval_kernels(const Problem& pr);
cudaError_t launch_swarm_init(const Problem& pr, const Swarm& sw,
                              const NodeDesc* nodes, int A, SwarmCoef co,
                              cudaStream_t st);
// z and ranges of every (tile, particle group); grid_cap = CTAs launched at
// most (the grid is persistent); pg = particles per group (0: pr.G's width);
// gather: read rows through pr.gidx from pr.Xg (when set) instead of pr.X.
// A > 0: the batch's node count (sw.pos holds A * pr.Pp rows); contiguous
// rows with d % 4 == 0 are then staged by tensor-map tile copies.
cudaError_t launch_project(const Problem& pr, const Swarm& sw,
                           const WorkTile* tiles, int n_tiles, int grid_cap,
                           cudaStream_t st, int pg = 0, bool gather = false, int A = 0);
// Whether k_project has a pg-particle group variant dividing pr.Pp.
bool project_group_ok(const Problem& pr, int pg);
// Cluster split S of the histogram kernel for A nodes of at most max_len
// entries on n_sm SMs, with clusters of at most max_cluster CTAs.
int hist_split(const Problem& pr, int A, int64_t max_len, int n_sm, int max_cluster);
// Largest power-of-two cluster size (<= 16) of the histogram kernel.
int hist_max_cluster(const Problem& pr);
// Scores of every (node, particle); bins_out[P, seg_len] (one node) or null.
// With do_update, also each particle's pbest step of iteration t.
cudaError_t launch_hist_scan(const Problem& pr, const Swarm& sw,
                             const NodeDesc* nodes, int A, int S,
                             int32_t* bins_out, int t, int do_update,
                             cudaStream_t st, const int32_t* list = nullptr);
// Histograms and scans of an FP32 search (no bins out, no top-k):
// classification (k_hist_cls) or the squared error (k_hist_mse), the same
// scores, pbest steps and move terms as launch_hist_scan, built for latency
// (see hist_kernels.cu). xtab: the device's c ln c table. hist_cls_fits:
// nodes of at most max_len entries stay within the regression kernel's
// 32-bit counters.
bool hist_cls_ok(const Problem& pr);
bool hist_cls_fits(const Problem& pr, int64_t max_len);
cudaError_t prepare_hist_cls(const Problem& pr);
int hist_cls_split(const Problem& pr, int A, int64_t max_len, int n_sm);
cudaError_t launch_hist_cls(const Problem& pr, const Swarm& sw, const NodeDesc* nodes, int A,
                            int S, int t, int do_update, const double* xtab, cudaStream_t st,
                            const int32_t* list = nullptr);
// Persistent search of classification nodes whose rows fit in shared memory:
// all T + 1 iterations in one launch, a cluster of S (1..8) CTAs per node of
// list[n_nodes] (A: the batch's node count, the gbest buffers' stride).
constexpr size_t kNodeSearchMaxSmem = 226 * 1024;
constexpr int kNodeThreads = 512;  // threads per CTA of the persistent search
// Dynamic shared memory of one CTA of an S-CTA cluster searching a node of
// n rows (SIZE_MAX when d is not a multiple of 4).
size_t node_search_smem(const Problem& pr, int n, int S);
cudaError_t launch_node_search(const Problem& pr, const Swarm& sw, const NodeDesc* nodes,
                               const int32_t* list, int n_nodes, int A, int S, size_t smem,
                               SwarmCoef co, cudaStream_t st);
// Small classification nodes: one warp per (node, particle) of the n_nodes
// nodes list[] names (scores, range reset and pbest step as k_hist_scan).
constexpr size_t kHistWarpMaxSmem = 160 * 1024;
bool hist_warp_ok(const Problem& pr);
cudaError_t launch_hist_warp(const Problem& pr, const Swarm& sw, const NodeDesc* nodes,
                             const int32_t* list, int n_nodes, int t, int do_update,
                             cudaStream_t st);
// Adaptive PSO step of each node after evaluation t (sw.apso; pr.P the
// swarm's particles, the elite candidate in slot pr.P): the gbest step, the
// elite candidate's acceptance (gB, or the worst particle's place), then
// for t < T the evolutionary factor of the current positions, the fuzzy
// state, the learning factors and inertia of the move to t + 1, and in the
// convergence state the next elite candidate, then the move of Eq. pso-1
// (k_move is not launched) (of the n_list nodes list[] names, when set).
cudaError_t launch_apso(const Problem& pr, const Swarm& sw, const NodeDesc* nodes, int A,
                        int t, SwarmCoef co, cudaStream_t st, const int32_t* list = nullptr,
                        int n_list = 0);
// The projection of iteration t with the swarm move folded in (classification
// or MSE searches in the FP32 form): for t > 0 every CTA first takes the gbest
// step of evaluation t - 1 of each node it projects (the rule of k_move) and
// forms the node's positions x_t = x + (ic + s2 (gB - x)) from pos_prev (the
// positions of t - 1) in shared memory; the CTA holding the node's first row
// tile writes x_t to sw.pos, v_t to sw.vel and the gbest records. Then z and
// the ranges of every (row tile, all particles) unit, as k_project (the same
// fused multiply-adds). tiles: for every node in order, for each of its
// step_slices(pr, sh) particle slices (WorkTile::pad = the slice's first
// particle), its step_rows(pr, sh)-row tiles; every node with at least one.
// sh picks the tile shape (0: the largest row tile with every particle;
// 1, 2: smaller row tiles; 3-5: the same with half the particles per unit;
// step_rows 0 when the swarm width has no such shape). The gbest step of
// the last evaluation is left to launch_move(t = T). With sw.node_step the
// histogram kernel has moved the swarm already: k_step loads the positions
// of t from pos_prev.
constexpr int kStepShapeCount = 6;
bool step_ok(const Problem& pr);
int step_rows(const Problem& pr, int sh);
int step_slices(const Problem& pr, int sh);
int step_grid(const Problem& pr, int sh, int n_sm);
cudaError_t prepare_step_kernels(const Problem& pr, int sh);
cudaError_t launch_step(const Problem& pr, const Swarm& sw, const float* pos_prev,
                        const NodeDesc* nodes, int A, const WorkTile* tiles, int n_tiles,
                        int grid, int sh, int t, cudaStream_t st);
// gbest step of iteration t and (t < T) the Eq. pso-1 move of every particle
// of A nodes to iteration t+1 (of the n_list nodes list[] names, when set).
cudaError_t launch_move(const Problem& pr, const Swarm& sw, const NodeDesc* nodes,
                        int A, int t, SwarmCoef co, cudaStream_t st,
                        const int32_t* list = nullptr, int n_list = 0);
// ---- probabilistic search (prob_kernels.cu; Sec. II-B) ---------------------
cudaError_t launch_prob_init(EvalRes* best, int32_t* best_idx, cudaStream_t st);
// Unit vectors e_{c0 + i} as rows i < count of pos[Pp, d], other rows zero.
cudaError_t launch_prob_units(int c0, int count, int Pp, int d, float* pos, cudaStream_t st);
// Candidates c0 .. c0 + count - 1 into pos[Pp, d] (rows past count zero) and
// all_pos[I, d]; rank_feat[d], w[d] (gamma^r), m[d] (floor(A_{r+1})).
cudaError_t launch_prob_candidates(uint64_t seed, uint32_t uid, int c0, int count, int Pp, int d,
                                   const int32_t* rank_feat, const double* w, const int32_t* m,
                                   int R, float* pos, float* all_pos, cudaStream_t st);
// Best so far after batch b (pr.P = the batch's candidates, scored in cur).
cudaError_t launch_prob_best(const Problem& pr, const EvalRes* cur, int c0, int b, EvalRes* best,
                             int32_t* best_idx, const float* all_pos, float* best_pos,
                             double* trace, EvalRes* all_scores, cudaStream_t st);
cudaError_t launch_prob_prune(int crit, int I, int d, const float* all_pos, const EvalRes* sc,
                              int q, int64_t cos_num, int64_t cos_den, uint8_t* pruned,
                              int32_t* kept, int32_t* n_kept, cudaStream_t st);

// ---- bfloat16 projection on the tensor cores (mma_kernels.cu) -------------
// Converts n_blocks blocks of R rows of src[*, d] (float, row stride d; rows
// at or past n_src_rows read as 0) to bfloat16 in the K-major, unswizzled
// core-matrix layout the MMA reads: block b, feature k, row r lives at
// element b*R*dp + (k/16)*R*16 + (r/8)*128 + ((k/8)&1)*64 + (r&7)*8 + (k&7).
cudaError_t launch_to_mma_layout(const float* src, int64_t n_src_rows, int d, int dp, int R,
                                 int64_t n_blocks, uint16_t* out, cudaStream_t st);
// Largest resident grid of k_project_mma for a problem (0 if it cannot run).
int mma_grid_cap(const Problem& pr, int n_sm);
cudaError_t prepare_mma_kernels(const Problem& pr);
// z and ranges of every (kMmaRows-row tile, all particles) with the BF16
// tensor-core MMA; posb[A, Pp*dp] in the MMA layout (R = Pp).
cudaError_t launch_project_mma(const Problem& pr, const Swarm& sw, const WorkTile* tiles,
                               int n_tiles, const uint16_t* posb, int grid,
                               cudaStream_t st);
// Writes the re-scored particles' scores cur2[A, kp] over sw.cur; with
// do_update, the pbest step of every particle and the gbest step of
// iteration t among the re-scored particles (Algorithm 1).
cudaError_t launch_merge(const Problem& pr, const Swarm& sw, int A, const EvalRes* cur2,
                         int kp, const int32_t* inv, int t, int do_update, cudaStream_t st);

// MSE moments of the entries of A nodes (tiles: kTS-row tiles with node
// index): per node the range of y and the weight W (acc_w[A], acc_y[A, 2]),
// then per entry m1 = round(w (y-c) 2^s), m2 = round(w (y-c)^2 2^(2s-t)),
// with c the node's mid-range and s, t chosen so each node sum stays below
// 2^61; mscale[A, 2] = 2^-s, 2^(t-2s).
cudaError_t launch_mse_moments(const Problem& pr, const WorkTile* tiles, int n_tiles, int A,
                               unsigned long long* acc_w, int32_t* acc_y, long long* m1,
                               long long* m2, double* mscale, cudaStream_t st);
cudaError_t launch_swarm_uniforms(uint64_t seed, uint32_t uid, uint32_t t,
                                  int P, int d, uint32_t purpose, float* u,
                                  cudaStream_t st);
cudaError_t launch_bootstrap(uint64_t seed, uint32_t tree, int64_t n,
                             uint32_t* w, cudaStream_t st);

}  // namespace slm

namespace slm {

// ---- tree-level kernels (tree_kernels.cu) ---------------------------------

// One node of the level being grown.
struct LevelNode {
  int32_t seg_start, seg_len;
  int32_t slot;   // tree * H + heap index
  int32_t depth;
};

struct TreeArrays {
  int32_t* kind;      // [T*H]
  float* dir;         // [T*H*d]
  float* zmin;        // [T*H]
  float* inv_w;
  int32_t* bin;
  int32_t* leaf_class;
  double* leaf_value;
  int64_t* weight;
  double* loss;
  int64_t* n_left;
  int64_t* n_right;
};

// Gathers rows / labels / targets of sample ids idx[E] into entry order:
// Xl[e] = X[idx[e]] (labels, y likewise; null arrays are skipped).
// Feature pre-screen: unit-vector positions of A nodes; the kept columns of
// each node's rows (feat[A][n], tiles of the nodes); gB lifted to d features.
cudaError_t launch_unit_positions(float* pos, int A, int Pp, int d, cudaStream_t st);
cudaError_t launch_range_reset(int32_t* zmm, int64_t count, cudaStream_t st);
cudaError_t launch_gather_cols(const float* X, int d, const int32_t* feat, int n,
                               const WorkTile* tiles, int n_tiles, float* Xs, cudaStream_t st);
cudaError_t launch_lift(const float* gs, const int32_t* feat, int A, int n, int d, float* gfull,
                        cudaStream_t st);
cudaError_t launch_gather(const float* X, const int32_t* labels, const float* y,
                          const int32_t* idx, int64_t E, int d, float* Xl,
                          int32_t* lab_l, float* y_l, cudaStream_t st);
// Per-node accumulators of the level statistics (zeroed before use, except
// ylo / yhi which start at INT_MAX / INT_MIN).
struct LevelAcc {
  unsigned long long* cls;  // [L, K] weighted class counts
  unsigned long long* w;    // [L] weight
  int32_t* ylo;             // [L] ordered-int target range (MSE)
  int32_t* yhi;
  double* tile_s;           // [n_tiles, 2] per-tile sum w y, sum w y^2
};
// Per-searched-node accumulators of the partition (zeroed before use).
struct PartAcc {
  unsigned long long* lk;   // [A, K] weighted left class counts
  unsigned long long* wl;   // [A] weighted left count
};
// Level arrays of one side of the ping-pong.
struct LevelArrays {
  float* X;
  int32_t* lab;
  float* y;
  uint32_t* w;
  int32_t* idx;
};

// Leaf fields of every level node, splittable[L], par[L*2] = parent
// (sum w y, sum w y^2). tiles / tile0: the level's kTS-row tiles, node l
// owning tiles [tile0[l], tile0[l+1]).
cudaError_t launch_node_stats(const Problem& pr, const LevelNode* nodes, int L,
                              const WorkTile* tiles, int n_tiles,
                              const int32_t* tile0, LevelAcc acc, TreeArrays tr,
                              int max_depth, double* par, int32_t* splittable,
                              cudaStream_t st);
// Side of each entry of the searched nodes' tiles under gB.
cudaError_t launch_partition(const Problem& pr, const Swarm& sw,
                             const WorkTile* tiles, int n_tiles, uint8_t* side,
                             int32_t* tile_left, PartAcc acc, cudaStream_t st);
// Per searched node: zero-gain test, tree fields, scatter bases.
// out3[A*3] = {split?, left entries, right entries}.
cudaError_t launch_decide(const Problem& pr, const Swarm& sw,
                          const NodeDesc* snodes, const int32_t* map,
                          const int32_t* tile0, int A, const int32_t* tile_left,
                          int32_t* tile_base, const unsigned long long* node_cls,
                          const double* par, PartAcc acc, TreeArrays tr,
                          int32_t* out3, int32_t* status, cudaStream_t st);
// Stable scatter of split nodes' entries into the next level's arrays.
// dst[A*2] = start of the left / right child segments (-1: not split).
cudaError_t launch_scatter(const Problem& pr, const WorkTile* tiles, int n_tiles,
                           const uint8_t* side, const int32_t* dst,
                           const int32_t* tile_base, const int32_t* tile0,
                           const int32_t* idx_cur, LevelArrays next,
                           cudaStream_t st);
// Root entries of bootstrap trees: for tree t, the samples with w > 0 in
// increasing order and their multiplicities, at offsets off[t]; counts[t].
cudaError_t launch_compact_nonzero(const uint32_t* w_all, int n_trees,
                                   int64_t n, int32_t* idx_out,
                                   uint32_t* w_out, const int64_t* off,
                                   int32_t* counts, cudaStream_t st);
// idx[c * stride + i] = i for i < n, c < copies.
cudaError_t launch_iota(int32_t* idx, int64_t n, int64_t stride, int copies,
                        cudaStream_t st);
// Checks labels in [0, K) and sample indices in [0, n); sets *status = 1 on
// the first violation.
cudaError_t launch_validate(const int32_t* labels, int64_t n, int K,
                            const int32_t* idx, int64_t n_idx,
                            int32_t* status, cudaStream_t st);
cudaError_t launch_predict(const float* X, int64_t n, int d, TreeArrays tr,
                           int n_trees, int H, int B, int K, int crit,
                           int32_t* class_out, double* value_out,
                           int32_t* leaf_out, cudaStream_t st);

// Boosting rounds: base = (float)(mean of y in double) and F[i] = base (one
// CTA, a fixed summation order); mean of (y - F)^2 in double (one CTA);
// r = y - F; F[i*K + k] += eta * (float)v_i; F = v; the softmax residuals
// R[k*n + i] = (float)([labels_i == k] - p_ik) (double); the mean
// cross-entropy (one CTA); the argmax of each row of F[n, K].
cudaError_t launch_boost_init(const float* y, int64_t n, float* F, float* base_out,
                              cudaStream_t st);
cudaError_t launch_boost_mse(const float* y, const float* F, int64_t n, double* out,
                             cudaStream_t st);
cudaError_t launch_boost_residual(const float* y, const float* F, float* r, int64_t n,
                                  cudaStream_t st);
cudaError_t launch_boost_update(float* F, const double* v, float eta, int64_t n,
                                cudaStream_t st, int K = 1, int k = 0);
cudaError_t launch_softmax_residual(const float* F, const int32_t* labels, int64_t n, int K,
                                    float* R, cudaStream_t st);
cudaError_t launch_boost_ce(const float* F, const int32_t* labels, int64_t n, int K,
                            double* out, cudaStream_t st);
cudaError_t launch_argmax_rows(const float* F, int64_t n, int K, int32_t* cls,
                               cudaStream_t st);
cudaError_t launch_fill_f(float* F, float v, int64_t n, cudaStream_t st);

// ---- learned swarm proposal (mlp_kernels.cu) --------------------------------

// Parameters, "input x output" row-major, FP32 masters and the bfloat16
// copies the network computes with.
struct MlpParams {
  float *W1, *b1, *W2, *b2, *W3, *b3;
  __nv_bfloat16 *W1b, *W2b, *W3b;
};
struct MlpGrads {
  float *W1, *b1, *W2, *b2, *W3, *b3;
};
// Adam moments of every parameter.
struct MlpState {
  float *mW1, *vW1, *mb1, *vb1, *mW2, *vW2, *mb2, *vb2, *mW3, *vW3, *mb3, *vb3;
};
// Activations of a batch of N samples: H1, H2, dH1, dH2 [N, H]; O, dO [N, OUT].
struct MlpWork {
  float *H1, *H2, *O, *dO, *dH1, *dH2;
};

// Network inputs of A nodes (entry-ordered rows of pr; K classes, or 4 y
// groups when pr.lab is null): stats[A, 5376]. Scratch: yr[A, 2],
// acc[A, K + 2, d], wk[A, K].
cudaError_t launch_node_stats(const Problem& pr, const NodeDesc* nodes, int A,
                              int64_t max_len, int K, int32_t* yr, double* acc, double* wk,
                              float* stats, int n_sm, cudaStream_t st);
cudaError_t launch_mlp_init(const MlpParams& m, uint64_t seed, cudaStream_t st);
cudaError_t launch_mlp_sync_bf16(const MlpParams& m, cudaStream_t st);
// w.O[N, OUT] = network(S[N, 5376]).
cudaError_t launch_mlp_forward(const MlpParams& m, const float* S, int N, MlpWork w,
                               cudaStream_t st);
// *loss = mean loss of the batch; g = its gradient (straight through the
// bfloat16 rounding of the weights).
cudaError_t launch_mlp_loss_grad(const MlpParams& m, const float* S, const int32_t* dims,
                                 const float* targets, int N, MlpWork w, MlpGrads g,
                                 double* loss, cudaStream_t st);
// Adam step t (beta 0.9 / 0.999, eps 1e-8) on every parameter; refreshes the
// bfloat16 copies.
cudaError_t launch_adam(MlpParams& m, MlpState& s, const MlpGrads& g, int t, float lr,
                        cudaStream_t st);
// dst[b, cols] = src rows idx[0..b).
cudaError_t launch_gather_rows(const float* src, int64_t cols, const int32_t* idx, int b,
                               float* dst, cudaStream_t st);
cudaError_t launch_gather_rows(const int32_t* src, int64_t cols, const int32_t* idx, int b,
                               int32_t* dst, cudaStream_t st);
// *acc += *v on the device.
cudaError_t launch_acc_double(double* acc, const double* v, cudaStream_t st);
// pos[P, d]: the seeded positions around mu_hat with radii rho[P].
cudaError_t launch_seed_positions(uint64_t seed, uint32_t uid, int P, int d,
                                  const float* mu_hat, const float* rho, float* pos,
                                  cudaStream_t st);
// Initial swarms of A nodes seeded from the network outputs prop[A, OUT].
cudaError_t launch_swarm_seed_init(const Problem& pr, const Swarm& sw, const NodeDesc* nodes,
                                   int A, SwarmCoef co, const float* prop, cudaStream_t st);

// ---- kernel attributes and occupancy, remembered per device --------------
// Searches plan their launches again at every level; the runtime calls that
// set a kernel's dynamic shared-memory limit or query its occupancy cost
// microseconds each, so their results are kept: a limit is raised only when
// a larger one is needed, an occupancy is queried once per (kernel, block,
// shared memory) that gives a nonzero answer.

struct KernelAttrCache {
  std::mutex mu;
  std::map<std::pair<int, const void*>, int> smem;      // largest limit set
  std::map<std::pair<int, const void*>, bool> cluster;  // non-portable sizes allowed
  std::map<std::tuple<int, const void*, int, size_t>, int> occ;
};

inline KernelAttrCache& kernel_attr_cache() {
  static KernelAttrCache c;
  return c;
}

// cudaFuncSetAttribute(fn, MaxDynamicSharedMemorySize, bytes) unless this
// device already allows fn at least bytes.
inline cudaError_t allow_smem(const void* fn, int bytes) {
  int dev = 0;
  if (cudaError_t e = cudaGetDevice(&dev)) return e;
  KernelAttrCache& c = kernel_attr_cache();
  {
    std::lock_guard<std::mutex> g(c.mu);
    const auto it = c.smem.find({dev, fn});
    if (it != c.smem.end() && it->second >= bytes) return cudaSuccess;
  }
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> g(c.mu);
    int& v = c.smem[{dev, fn}];
    if (bytes > v) v = bytes;
  }
  return e;
}

// cudaFuncSetAttribute(fn, NonPortableClusterSizeAllowed, 1), once per device.
inline cudaError_t allow_cluster(const void* fn) {
  int dev = 0;
  if (cudaError_t e = cudaGetDevice(&dev)) return e;
  KernelAttrCache& c = kernel_attr_cache();
  {
    std::lock_guard<std::mutex> g(c.mu);
    if (c.cluster.count({dev, fn})) return cudaSuccess;
  }
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> g(c.mu);
    c.cluster[{dev, fn}] = true;
  }
  return e;
}

// cudaOccupancyMaxActiveBlocksPerMultiprocessor, remembered per device.
inline cudaError_t occupancy(int* per_sm, const void* fn, int threads, size_t smem) {
  int dev = 0;
  if (cudaError_t e = cudaGetDevice(&dev)) return e;
  KernelAttrCache& c = kernel_attr_cache();
  const auto key = std::make_tuple(dev, fn, threads, smem);
  {
    std::lock_guard<std::mutex> g(c.mu);
    const auto it = c.occ.find(key);
    if (it != c.occ.end()) {
      *per_sm = it->second;
      return cudaSuccess;
    }
  }
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, threads, smem);
  if (e == cudaSuccess && *per_sm > 0) {  // (zero: perhaps a limit not yet raised)
    std::lock_guard<std::mutex> g(c.mu);
    c.occ[key] = *per_sm;
  }
  return e;
}

}  // namespace slm
