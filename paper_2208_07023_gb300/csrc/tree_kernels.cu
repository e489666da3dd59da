// Tree-level kernels: node statistics, partition of searched nodes, stable
// scatter into the next level, gathers, bootstrap bags, prediction.
//
// Algorithm 2: a node that meets the split condition is searched, split on
// gB, and its two children are grown next; otherwise it becomes a leaf.
// Sec. II-A: leaves predict their majority class (ties: lowest class id);
// regression leaves predict the mean target. The split sets are Eqs. (3)-(4):
// right ("+") iff bin(gB . x) >= b*, i.e. z >= t_b.
//
// Every per-level pass runs over the same kTS-row tiles of the entry-ordered
// level arrays (one CTA per tile), followed by a one-thread-per-node kernel
// where a per-node decision is needed, so shallow levels with a few large
// nodes keep the whole GPU busy.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>

#include "slm_internal.cuh"

namespace slm {

namespace {

constexpr int kTT = kTS;  // threads per CTA = rows per tile

__device__ __forceinline__ int bin_of(float z, float zmin, float inv_w, int B) {
  const float off = __fsub_rn(z, zmin);
  const float pos = __fmul_rn(off, inv_w);
  int b = (int)floorf(pos);
  b = b > B - 1 ? B - 1 : b;
  return b < 0 ? 0 : b;
}

__device__ __forceinline__ int f2ord(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}

// gB . x as one fmaf per feature in increasing order from +0, the same
// sequence the scoring kernels run.
__device__ __forceinline__ float project_row(const float* __restrict__ x,
                                             const float* __restrict__ g, int d) {
  float acc = 0.0f;
  for (int j = 0; j < d; ++j) acc = fmaf(__ldg(x + j), g[j], acc);
  return acc;
}

// Block-wide exclusive scan of one int per thread (kTT threads); returns the
// prefix, *total = block sum.
__device__ __forceinline__ int block_excl_scan(int v, int* total, int* sbuf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += u;
  }
  __syncthreads();
  if (lane == 31) sbuf[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int wv = lane < kTT / 32 ? sbuf[lane] : 0;
    int wi = wv;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, wi, off);
      if (lane >= off) wi += u;
    }
    if (lane < kTT / 32) sbuf[lane] = wi - wv;
    if (lane == kTT / 32 - 1) sbuf[kTT / 32] = wi;
  }
  __syncthreads();
  *total = sbuf[kTT / 32];
  return sbuf[warp] + incl - v;
}

// ---- node statistics (per tile, then per node) ------------------------------------

// Per tile of a level node: weighted class counts and weight (integer global
// atomics: order-free), target range (ordered-int atomics) and the tile's
// partial target sums (summed per node in tile order by k_stats_finish).
__global__ void __launch_bounds__(kTT)
    k_stats_tiles(Problem pr, const WorkTile* __restrict__ tiles, LevelAcc acc) {
  const WorkTile wt = tiles[blockIdx.x];
  const int K = pr.K;
  __shared__ unsigned long long s_cnt[kMaxClasses];
  __shared__ unsigned long long s_w;
  __shared__ double s_sy[kTT], s_sq[kTT];
  __shared__ int s_lo, s_hi;
  if (threadIdx.x < kMaxClasses) s_cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    s_w = 0;
    s_lo = INT_MAX;
    s_hi = INT_MIN;
  }
  __syncthreads();
  const int r = threadIdx.x;
  double sy = 0.0, sq = 0.0;
  if (r < wt.rows) {
    const int64_t e = (int64_t)wt.row0 + r;
    const uint32_t w = pr.w ? pr.w[e] : 1u;
    atomicAdd(&s_w, (unsigned long long)w);
    if (pr.crit == SLM_MSE) {
      const float yv = pr.y[e];
      sy = (double)w * (double)yv;
      sq = sy * (double)yv;
      atomicMin(&s_lo, f2ord(yv));
      atomicMax(&s_hi, f2ord(yv));
    } else {
      atomicAdd(&s_cnt[pr.lab[e]], (unsigned long long)w);
    }
  }
  s_sy[threadIdx.x] = sy;
  s_sq[threadIdx.x] = sq;
  __syncthreads();
  for (int off = kTT / 2; off > 0; off >>= 1) {  // fixed order: deterministic
    if (threadIdx.x < off) {
      s_sy[threadIdx.x] += s_sy[threadIdx.x + off];
      s_sq[threadIdx.x] += s_sq[threadIdx.x + off];
    }
    __syncthreads();
  }
  const int l = wt.node;
  if (threadIdx.x < K && pr.crit != SLM_MSE && s_cnt[threadIdx.x])
    atomicAdd(&acc.cls[(int64_t)l * K + threadIdx.x], s_cnt[threadIdx.x]);
  if (threadIdx.x == 0) {
    atomicAdd(&acc.w[l], s_w);
    acc.tile_s[2 * blockIdx.x] = s_sy[0];
    acc.tile_s[2 * blockIdx.x + 1] = s_sq[0];
    if (pr.crit == SLM_MSE && s_lo != INT_MAX) {
      atomicMin(&acc.ylo[l], s_lo);
      atomicMax(&acc.yhi[l], s_hi);
    }
  }
}

// One thread per level node: leaf value, splittable flag, parent sums.
__global__ void k_stats_finish(Problem pr, const LevelNode* __restrict__ nodes,
                               const int32_t* __restrict__ tile0, int L, LevelAcc acc,
                               TreeArrays tr, int max_depth, double* par,
                               int32_t* splittable) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  const LevelNode nd = nodes[l];
  const int K = pr.K;
  const unsigned long long nw = acc.w[l];
  const int slot = nd.slot;
  bool pure;
  if (pr.crit == SLM_MSE) {
    double sy = 0.0, sq = 0.0;
    for (int t = tile0[l]; t < tile0[l + 1]; ++t) {
      sy += acc.tile_s[2 * t];
      sq += acc.tile_s[2 * t + 1];
    }
    tr.leaf_value[slot] = nw ? sy / (double)nw : 0.0;
    tr.leaf_class[slot] = -1;
    pure = !(acc.yhi[l] > acc.ylo[l]);
    par[2 * l] = sy;
    par[2 * l + 1] = sq;
  } else {
    int best = 0, nonzero = 0;
    const unsigned long long* c = acc.cls + (int64_t)l * K;
    for (int k = 0; k < K; ++k) {
      if (c[k] > c[best]) best = k;
      nonzero += c[k] > 0;
    }
    tr.leaf_class[slot] = best;
    tr.leaf_value[slot] = 0.0;
    pure = nonzero <= 1;
  }
  tr.kind[slot] = 0;
  tr.weight[slot] = (int64_t)nw;
  tr.bin[slot] = -1;
  splittable[l] = (nd.depth < max_depth) && nw >= 2ull * (unsigned long long)pr.min_leaf &&
                  !pure;
}

// ---- partition (per tile), decision (per node), scatter (per tile) --------------

// Side of every entry of a searched node's tile under its gB: right iff
// bin(gB . x) >= b*. Stores the tile's left-entry count; adds the node's left
// weight and left class counts.
__global__ void __launch_bounds__(kTT)
    k_part_tiles(Problem pr, Swarm sw, const WorkTile* __restrict__ tiles, uint8_t* side,
                 int32_t* tile_left, PartAcc acc) {
  const WorkTile wt = tiles[blockIdx.x];
  const int a = wt.node;
  const EvalRes gb = sw.gb[a];
  const int d = pr.d, K = pr.K;
  extern __shared__ float s_g[];  // [d]
  __shared__ unsigned long long s_lk[kMaxClasses];
  __shared__ unsigned long long s_wl;
  __shared__ int s_n;
  if (!gb.valid) {
    if (threadIdx.x == 0) tile_left[blockIdx.x] = 0;
    return;
  }
  for (int j = threadIdx.x; j < d; j += kTT) s_g[j] = sw.gbest[(int64_t)a * d + j];
  if (threadIdx.x < kMaxClasses) s_lk[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    s_wl = 0;
    s_n = 0;
  }
  __syncthreads();
  const int r = threadIdx.x;
  if (r < wt.rows) {
    const int64_t e = (int64_t)wt.row0 + r;
    const float z = project_row(pr.X + e * d, s_g, d);
    const int b = bin_of(z, gb.zmin, gb.inv_w, pr.B);
    const int right = b >= gb.bin;
    side[e] = (uint8_t)right;
    if (!right) {
      const uint32_t w = pr.w ? pr.w[e] : 1u;
      atomicAdd(&s_n, 1);
      atomicAdd(&s_wl, (unsigned long long)w);
      if (pr.crit != SLM_MSE) atomicAdd(&s_lk[pr.lab[e]], (unsigned long long)w);
    }
  }
  __syncthreads();
  if (threadIdx.x < K && pr.crit != SLM_MSE && s_lk[threadIdx.x])
    atomicAdd(&acc.lk[(int64_t)a * K + threadIdx.x], s_lk[threadIdx.x]);
  if (threadIdx.x == 0) {
    tile_left[blockIdx.x] = s_n;
    if (s_wl) atomicAdd(&acc.wl[a], s_wl);
  }
}

// One thread per searched node: zero-gain test, internal-node fields, tile
// bases of the scatter. out3[a] = {split?, left entries, right entries}.
__global__ void k_decide(Problem pr, Swarm sw, const NodeDesc* __restrict__ snodes,
                         const int32_t* __restrict__ map, const int32_t* __restrict__ tile0,
                         int A, const int32_t* __restrict__ tile_left, int32_t* tile_base,
                         const unsigned long long* __restrict__ node_cls,
                         const double* __restrict__ par, PartAcc acc, TreeArrays tr,
                         int32_t* out3, int32_t* status) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A) return;
  const NodeDesc nd = snodes[a];
  const EvalRes gb = sw.gb[a];
  const int d = pr.d, K = pr.K;
  int nl_entries = 0;
  for (int t = tile0[a]; t < tile0[a + 1]; ++t) {
    tile_base[t] = nl_entries;
    nl_entries += gb.valid ? tile_left[t] : 0;
  }
  out3[3 * a + 1] = nl_entries;
  out3[3 * a + 2] = nd.seg_len - nl_entries;
  if (!gb.valid) {
    out3[3 * a] = 0;
    return;
  }
  const int l = map[a];
  const unsigned long long wleft = acc.wl[a];
  const unsigned long long nw = (unsigned long long)(gb.nl + gb.nr);
  if (wleft != (unsigned long long)gb.nl) atomicExch(status, 2);  // must agree
  // Zero gain: children keep the parent's class mix (Gini and entropy are
  // strictly concave), or the MSE does not drop below the parent's.
  bool no_gain;
  if (pr.crit == SLM_MSE) {
    const double sy = par[2 * l], sq = par[2 * l + 1];
    const double parent = (sq - sy * sy / (double)nw) / (double)nw;
    no_gain = !(gb.loss < parent);
  } else {
    no_gain = true;
    for (int k = 0; k < K; ++k)
      if (acc.lk[(int64_t)a * K + k] * nw != node_cls[(int64_t)l * K + k] * wleft)
        no_gain = false;
  }
  out3[3 * a] = no_gain ? 0 : 1;
  if (no_gain) return;
  const int slot = nd.slot;
  tr.kind[slot] = 1;
  for (int j = 0; j < d; ++j) tr.dir[(int64_t)slot * d + j] = sw.gbest[(int64_t)a * d + j];
  tr.zmin[slot] = gb.zmin;
  tr.inv_w[slot] = gb.inv_w;
  tr.bin[slot] = gb.bin;
  tr.loss[slot] = gb.loss;
  tr.n_left[slot] = gb.nl;
  tr.n_right[slot] = gb.nr;
}

// Stable scatter of a split node's tile into its children's segments:
// rows, labels / targets, multiplicities and sample ids.
__global__ void __launch_bounds__(kTT)
    k_scatter(Problem pr, const WorkTile* __restrict__ tiles, const uint8_t* __restrict__ side,
              const int32_t* __restrict__ dst, const int32_t* __restrict__ tile_base,
              const int32_t* __restrict__ tile0, const int32_t* __restrict__ idx_cur,
              LevelArrays nx) {
  const WorkTile wt = tiles[blockIdx.x];
  const int a = wt.node;
  const int dl = dst[2 * a], dr = dst[2 * a + 1];
  if (dl < 0) return;
  const int d = pr.d;
  __shared__ int sbuf[kTT / 32 + 1];
  __shared__ int s_dst[kTT];
  const int r = threadIdx.x;
  const bool in = r < wt.rows;
  const int64_t e = (int64_t)wt.row0 + r;
  const int is_left = in && !side[e];
  int tot_l;
  const int rank_l = block_excl_scan(is_left, &tot_l, sbuf);
  const int base_l = tile_base[blockIdx.x];
  const int rows_before = ((int)blockIdx.x - tile0[a]) * kTS;  // full tiles
  const int base_r = rows_before - base_l;
  if (in) {
    const int32_t pos = is_left ? dl + base_l + rank_l : dr + base_r + (r - rank_l);
    s_dst[r] = pos;
    nx.idx[pos] = idx_cur[e];
    if (nx.lab) nx.lab[pos] = pr.lab[e];
    if (nx.y) nx.y[pos] = pr.y[e];
    if (nx.w) nx.w[pos] = pr.w[e];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < wt.rows * d; q += kTT) {
    const int rr = q / d, j = q - rr * d;
    nx.X[(int64_t)s_dst[rr] * d + j] = pr.X[((int64_t)wt.row0 + rr) * d + j];
  }
}

__global__ void __launch_bounds__(kTT)
    k_compact_nonzero(const uint32_t* __restrict__ w_all, int64_t n, int32_t* idx_out,
                      uint32_t* w_out, const int64_t* __restrict__ off, int32_t* counts) {
  const int t = blockIdx.x;
  const uint32_t* w = w_all + (int64_t)t * n;
  __shared__ int sbuf[kTT / 32 + 1];
  const int64_t base = off[t];
  int count = 0;
  for (int64_t s0 = 0; s0 < n; s0 += kTT) {
    const int64_t s = s0 + threadIdx.x;
    const uint32_t ws = s < n ? w[s] : 0u;
    const int nz = ws > 0;
    int tot;
    const int rank = block_excl_scan(nz, &tot, sbuf);
    if (nz) {
      idx_out[base + count + rank] = (int32_t)s;
      w_out[base + count + rank] = ws;
    }
    count += tot;
  }
  if (threadIdx.x == 0) counts[t] = count;
}

__global__ void k_gather(const float* __restrict__ X, const int32_t* __restrict__ labels,
                         const float* __restrict__ y, const int32_t* __restrict__ idx,
                         int64_t E, int d, float* Xl, int32_t* lab_l, float* y_l) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= E * d) return;
  const int64_t e = q / d;
  const int j = (int)(q - e * d);
  const int64_t s = idx[e];
  Xl[q] = X[s * d + j];
  if (j == 0) {
    if (lab_l) lab_l[e] = labels[s];
    if (y_l) y_l[e] = y[s];
  }
}

// idx[c * stride + i] = i for i < n, c < copies.
__global__ void k_iota(int32_t* idx, int64_t n, int64_t stride, int copies) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * copies) return;
  const int64_t cpy = i / n, r = i - cpy * n;
  idx[cpy * stride + r] = (int32_t)r;
}

__global__ void k_validate(const int32_t* labels, int64_t n, int K, const int32_t* idx,
                           int64_t n_idx, int32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (labels && i < n) {
    const int32_t c = labels[i];
    if (c < 0 || c >= K) atomicExch(status, 1);
  }
  if (idx && i < n_idx) {
    const int32_t s = idx[i];
    if (s < 0 || (int64_t)s >= n) atomicExch(status, 1);
  }
}

__global__ void k_predict(const float* __restrict__ X, int64_t n, int d, TreeArrays tr,
                          int n_trees, int H, int B, int K, int crit, int32_t* class_out,
                          double* value_out, int32_t* leaf_out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float* x = X + s * d;
  int votes[kMaxClasses];
  for (int k = 0; k < kMaxClasses; ++k) votes[k] = 0;
  double vsum = 0.0;
  for (int t = 0; t < n_trees; ++t) {
    const int64_t base = (int64_t)t * H;
    int h = 0;
    while (h < H && tr.kind[base + h] == 1) {
      const int64_t slot = base + h;
      const float* g = tr.dir + slot * d;
      float acc = 0.0f;
      for (int j = 0; j < d; ++j) acc = fmaf(__ldg(x + j), __ldg(g + j), acc);
      const int b = bin_of(acc, tr.zmin[slot], tr.inv_w[slot], B);
      h = b >= tr.bin[slot] ? 2 * h + 2 : 2 * h + 1;
    }
    if (leaf_out) leaf_out[s * n_trees + t] = h;
    if (crit == SLM_MSE)
      vsum += tr.leaf_value[base + h];
    else
      votes[tr.leaf_class[base + h]] += 1;
  }
  if (crit == SLM_MSE) {
    if (value_out) value_out[s] = vsum / (double)n_trees;
    if (class_out) class_out[s] = -1;
  } else {
    int best = 0;
    for (int k = 1; k < K; ++k)
      if (votes[k] > votes[best]) best = k;
    if (class_out) class_out[s] = best;
    if (value_out) value_out[s] = (double)best;
  }
}


// ---- feature pre-screen (Sec. III-B, Algorithm 2) --------------------------------

// pos[a][p][j] = 1 if p == j else 0: particle k of every node is the unit
// vector e_k (its projection is feature k itself).
__global__ void k_unit_positions(float* pos, int A, int Pp, int d) {
  const int64_t total = (int64_t)A * Pp * d;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pj = i % ((int64_t)Pp * d);
    pos[i] = (pj / d == pj % d) ? 1.0f : 0.0f;
  }
}

// zmm[i] = (INT_MAX, INT_MIN): empty ordered-int ranges.
__global__ void k_range_reset(int32_t* zmm, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    zmm[2 * i] = INT_MAX;
    zmm[2 * i + 1] = INT_MIN;
  }
}

// Xs[e][j] = X[e][feat[a][j]] for the rows of each tile of node a.
__global__ void k_gather_cols(const float* __restrict__ X, int d,
                              const int32_t* __restrict__ feat, int n,
                              const WorkTile* __restrict__ tiles, float* Xs) {
  const WorkTile wt = tiles[blockIdx.x];
  const int32_t* f = feat + (int64_t)wt.node * n;
  for (int i = threadIdx.x; i < wt.rows * n; i += blockDim.x) {
    const int r = i / n, j = i - r * n;
    const int64_t e = (int64_t)wt.row0 + r;
    Xs[e * n + j] = X[e * d + f[j]];
  }
}

// gfull[a][k] = gs[a][j] where feat[a][j] = k, else 0.
__global__ void k_lift(const float* __restrict__ gs, const int32_t* __restrict__ feat, int n,
                       int d, float* gfull) {
  const int a = blockIdx.x;
  for (int k = threadIdx.x; k < d; k += blockDim.x) gfull[(int64_t)a * d + k] = 0.0f;
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    gfull[(int64_t)a * d + feat[(int64_t)a * n + j]] = gs[(int64_t)a * n + j];
}

}  // namespace

cudaError_t launch_node_stats(const Problem& pr, const LevelNode* nodes, int L,
                              const WorkTile* tiles, int n_tiles, const int32_t* tile0,
                              LevelAcc acc, TreeArrays tr, int max_depth, double* par,
                              int32_t* splittable, cudaStream_t st) {
  if (L <= 0) return cudaSuccess;
  if (n_tiles > 0) k_stats_tiles<<<n_tiles, kTT, 0, st>>>(pr, tiles, acc);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  k_stats_finish<<<(L + 127) / 128, 128, 0, st>>>(pr, nodes, tile0, L, acc, tr, max_depth,
                                                  par, splittable);
  return cudaGetLastError();
}

cudaError_t launch_partition(const Problem& pr, const Swarm& sw, const WorkTile* tiles,
                             int n_tiles, uint8_t* side, int32_t* tile_left, PartAcc acc,
                             cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  k_part_tiles<<<n_tiles, kTT, sizeof(float) * pr.d, st>>>(pr, sw, tiles, side, tile_left,
                                                            acc);
  return cudaGetLastError();
}

cudaError_t launch_decide(const Problem& pr, const Swarm& sw, const NodeDesc* snodes,
                          const int32_t* map, const int32_t* tile0, int A,
                          const int32_t* tile_left, int32_t* tile_base,
                          const unsigned long long* node_cls, const double* par,
                          PartAcc acc, TreeArrays tr, int32_t* out3, int32_t* status,
                          cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  k_decide<<<(A + 127) / 128, 128, 0, st>>>(pr, sw, snodes, map, tile0, A, tile_left,
                                            tile_base, node_cls, par, acc, tr, out3, status);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const Problem& pr, const WorkTile* tiles, int n_tiles,
                           const uint8_t* side, const int32_t* dst, const int32_t* tile_base,
                           const int32_t* tile0, const int32_t* idx_cur, LevelArrays next,
                           cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  k_scatter<<<n_tiles, kTT, 0, st>>>(pr, tiles, side, dst, tile_base, tile0, idx_cur, next);
  return cudaGetLastError();
}

cudaError_t launch_compact_nonzero(const uint32_t* w_all, int n_trees, int64_t n,
                                   int32_t* idx_out, uint32_t* w_out, const int64_t* off,
                                   int32_t* counts, cudaStream_t st) {
  if (n_trees <= 0) return cudaSuccess;
  k_compact_nonzero<<<n_trees, kTT, 0, st>>>(w_all, n, idx_out, w_out, off, counts);
  return cudaGetLastError();
}

cudaError_t launch_gather(const float* X, const int32_t* labels, const float* y,
                          const int32_t* idx, int64_t E, int d, float* Xl, int32_t* lab_l,
                          float* y_l, cudaStream_t st) {
  const int64_t total = E * d;
  if (total <= 0) return cudaSuccess;
  k_gather<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(X, labels, y, idx, E, d, Xl,
                                                           lab_l, y_l);
  return cudaGetLastError();
}

cudaError_t launch_iota(int32_t* idx, int64_t n, int64_t stride, int copies,
                        cudaStream_t st) {
  const int64_t total = n * copies;
  if (total <= 0) return cudaSuccess;
  k_iota<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(idx, n, stride, copies);
  return cudaGetLastError();
}

cudaError_t launch_validate(const int32_t* labels, int64_t n, int K, const int32_t* idx,
                            int64_t n_idx, int32_t* status, cudaStream_t st) {
  const int64_t m = (labels && n > n_idx) ? n : n_idx;
  if (m <= 0) return cudaSuccess;
  k_validate<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(labels, n, K, idx, n_idx, status);
  return cudaGetLastError();
}

cudaError_t launch_predict(const float* X, int64_t n, int d, TreeArrays tr, int n_trees,
                           int H, int B, int K, int crit, int32_t* class_out,
                           double* value_out, int32_t* leaf_out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_predict<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(X, n, d, tr, n_trees, H, B, K, crit,
                                                        class_out, value_out, leaf_out);
  return cudaGetLastError();
}

cudaError_t launch_unit_positions(float* pos, int A, int Pp, int d, cudaStream_t st) {
  const int64_t total = (int64_t)A * Pp * d;
  if (total <= 0) return cudaSuccess;
  const int64_t blocks = (total + 255) / 256;
  k_unit_positions<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, st>>>(pos, A, Pp, d);
  return cudaGetLastError();
}

cudaError_t launch_range_reset(int32_t* zmm, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int64_t blocks = (count + 255) / 256;
  k_range_reset<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, st>>>(zmm, count);
  return cudaGetLastError();
}

cudaError_t launch_gather_cols(const float* X, int d, const int32_t* feat, int n,
                               const WorkTile* tiles, int n_tiles, float* Xs, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  k_gather_cols<<<(unsigned)n_tiles, 256, 0, st>>>(X, d, feat, n, tiles, Xs);
  return cudaGetLastError();
}

cudaError_t launch_lift(const float* gs, const int32_t* feat, int A, int n, int d, float* gfull,
                        cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  k_lift<<<(unsigned)A, 256, 0, st>>>(gs, feat, n, d, gfull);
  return cudaGetLastError();
}

// ---- SLR Boost: the boosting rounds' elementwise steps --------------------------

namespace {

constexpr int kBoostThreads = 1024;

// Sum over one CTA of kBoostThreads in a fixed order: per thread in stride
// order (done by the caller), then a shuffle tree per warp, then warp 0 over
// the warps' sums. Thread 0 returns the total.
__device__ double boost_block_sum(double v) {
  __shared__ double sh[kBoostThreads / 32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  v = threadIdx.x < kBoostThreads / 32 ? sh[threadIdx.x] : 0.0;
  if (threadIdx.x < 32)
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// base = (float)(mean of y), summed in double; F[i] = base.
__global__ void __launch_bounds__(kBoostThreads)
    k_boost_init(const float* __restrict__ y, int64_t n, float* F, float* base_out) {
  __shared__ float s_base;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kBoostThreads) s += (double)y[i];
  s = boost_block_sum(s);
  if (threadIdx.x == 0) {
    s_base = (float)(s / (double)n);
    *base_out = s_base;
  }
  __syncthreads();
  const float b = s_base;
  for (int64_t i = threadIdx.x; i < n; i += kBoostThreads) F[i] = b;
}

// Mean over i of (y_i - F_i)^2 in double.
__global__ void __launch_bounds__(kBoostThreads)
    k_boost_mse(const float* __restrict__ y, const float* __restrict__ F, int64_t n,
                double* out) {
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kBoostThreads) {
    const double di = (double)y[i] - (double)F[i];
    s += di * di;
  }
  s = boost_block_sum(s);
  if (threadIdx.x == 0) *out = s / (double)n;
}

__global__ void k_boost_residual(const float* __restrict__ y, const float* __restrict__ F,
                                 float* r, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = __fsub_rn(y[i], F[i]);
}

// F[i*K + k] += eta * (float)v_i, one rounding per operation.
__global__ void k_boost_update(float* F, const double* __restrict__ v, float eta, int64_t n,
                               int K, int k) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    F[i * K + k] = __fadd_rn(F[i * K + k], __fmul_rn(eta, (float)v[i]));
}

// Softmax of one row of K scores in double: its maximum and the sum of
// exp(F_k - max) over k ascending.
__device__ __forceinline__ void softmax_row(const float* f, int K, double* mx, double* s) {
  double m = (double)f[0];
  for (int k = 1; k < K; ++k) m = (double)f[k] > m ? (double)f[k] : m;
  double t = 0.0;
  for (int k = 0; k < K; ++k) t += exp((double)f[k] - m);
  *mx = m;
  *s = t;
}

// R[k*n + i] = (float)([labels_i == k] - p_ik), p the softmax of F's row i.
__global__ void k_softmax_residual(const float* __restrict__ F, const int32_t* __restrict__ lab,
                                   int64_t n, int K, float* R) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float* f = F + i * K;
    double mx, sum;
    softmax_row(f, K, &mx, &sum);
    const int y = lab[i];
    for (int k = 0; k < K; ++k)
      R[(int64_t)k * n + i] = (float)((y == k ? 1.0 : 0.0) - exp((double)f[k] - mx) / sum);
  }
}

// Mean over i of -log p_{i, labels_i} (log-sum-exp form) in double.
__global__ void __launch_bounds__(kBoostThreads)
    k_boost_ce(const float* __restrict__ F, const int32_t* __restrict__ lab, int64_t n, int K,
               double* out) {
  double t = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kBoostThreads) {
    const float* f = F + i * K;
    double mx, sum;
    softmax_row(f, K, &mx, &sum);
    t += -(((double)f[lab[i]] - mx) - log(sum));
  }
  t = boost_block_sum(t);
  if (threadIdx.x == 0) *out = t / (double)n;
}

// class_out[i] = argmax over k of F[i*K + k], ties to the lower class.
__global__ void k_argmax_rows(const float* __restrict__ F, int64_t n, int K, int32_t* cls) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float* f = F + i * K;
    int b = 0;
    for (int k = 1; k < K; ++k)
      if (f[k] > f[b]) b = k;
    cls[i] = b;
  }
}

__global__ void k_fill_f(float* F, float v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    F[i] = v;
}

unsigned elementwise_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_boost_init(const float* y, int64_t n, float* F, float* base_out,
                              cudaStream_t st) {
  if (n <= 0) return cudaErrorInvalidValue;
  k_boost_init<<<1, kBoostThreads, 0, st>>>(y, n, F, base_out);
  return cudaGetLastError();
}

cudaError_t launch_boost_mse(const float* y, const float* F, int64_t n, double* out,
                             cudaStream_t st) {
  if (n <= 0) return cudaErrorInvalidValue;
  k_boost_mse<<<1, kBoostThreads, 0, st>>>(y, F, n, out);
  return cudaGetLastError();
}

cudaError_t launch_boost_residual(const float* y, const float* F, float* r, int64_t n,
                                  cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_boost_residual<<<elementwise_blocks(n), 256, 0, st>>>(y, F, r, n);
  return cudaGetLastError();
}

cudaError_t launch_boost_update(float* F, const double* v, float eta, int64_t n,
                                cudaStream_t st, int K, int k) {
  if (n <= 0) return cudaSuccess;
  k_boost_update<<<elementwise_blocks(n), 256, 0, st>>>(F, v, eta, n, K, k);
  return cudaGetLastError();
}

cudaError_t launch_softmax_residual(const float* F, const int32_t* labels, int64_t n, int K,
                                    float* R, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_softmax_residual<<<elementwise_blocks(n), 256, 0, st>>>(F, labels, n, K, R);
  return cudaGetLastError();
}

cudaError_t launch_boost_ce(const float* F, const int32_t* labels, int64_t n, int K,
                            double* out, cudaStream_t st) {
  if (n <= 0) return cudaErrorInvalidValue;
  k_boost_ce<<<1, kBoostThreads, 0, st>>>(F, labels, n, K, out);
  return cudaGetLastError();
}

cudaError_t launch_argmax_rows(const float* F, int64_t n, int K, int32_t* cls,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_argmax_rows<<<elementwise_blocks(n), 256, 0, st>>>(F, n, K, cls);
  return cudaGetLastError();
}

cudaError_t launch_fill_f(float* F, float v, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_fill_f<<<elementwise_blocks(n), 256, 0, st>>>(F, v, n);
  return cudaGetLastError();
}

}  // namespace slm
