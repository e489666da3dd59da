// Tree-level kernels: node statistics, partition of searched nodes, stable
// compaction into the next level, bootstrap bags, prediction.
//
// Algorithm 2: a node that meets the split condition is searched, split on
// gB, and its two children are grown next; otherwise it becomes a leaf.
// Sec. II-A: leaves predict their majority class (ties: lowest class id);
// regression leaves predict the mean target. The split sets are Eqs. (3)-(4):
// right ("+") iff bin(gB . x) >= b*, i.e. z >= t_b.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>

#include "slm_internal.cuh"

namespace slm {

namespace {

constexpr int kTT = 256;  // threads per CTA

__device__ __forceinline__ int bin_of(float z, float zmin, float inv_w, int B) {
  const float off = __fsub_rn(z, zmin);
  const float pos = __fmul_rn(off, inv_w);
  int b = (int)floorf(pos);
  b = b > B - 1 ? B - 1 : b;
  return b < 0 ? 0 : b;
}

// gB . x as one fmaf per feature in increasing order from +0, the same
// sequence the scoring kernels run.
__device__ __forceinline__ float project_row(const float* __restrict__ x,
                                             const float* __restrict__ g,
                                             int d) {
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
    int wv = lane < kTT / 32 ? sbuf[lane] : 0;
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

__global__ void __launch_bounds__(kTT)
    k_node_stats(Problem pr, const LevelNode* __restrict__ nodes,
                 TreeArrays tr, int max_depth, uint32_t* cls, double* par,
                 int32_t* splittable) {
  const int l = blockIdx.x;
  const LevelNode nd = nodes[l];
  __shared__ unsigned long long s_cnt[kMaxClasses];
  __shared__ unsigned long long s_w;
  __shared__ double s_sy[kTT], s_sq[kTT];
  __shared__ float s_lo[kTT], s_hi[kTT];
  const int K = pr.K;
  if (threadIdx.x < kMaxClasses) s_cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_w = 0;
  __syncthreads();
  unsigned long long wsum = 0;
  double sy = 0.0, sq = 0.0;
  float lo = INFINITY, hi = -INFINITY;
  for (int r = threadIdx.x; r < nd.seg_len; r += kTT) {
    const int64_t e = (int64_t)nd.seg_start + r;
    const uint32_t w = pr.w ? pr.w[e] : 1u;
    wsum += w;
    if (pr.crit == SLM_MSE) {
      const float yv = pr.y[e];
      const double wy = (double)w * (double)yv;
      sy += wy;
      sq += wy * (double)yv;
      lo = fminf(lo, yv);
      hi = fmaxf(hi, yv);
    } else {
      atomicAdd(&s_cnt[pr.lab[e]], (unsigned long long)w);
    }
  }
  atomicAdd(&s_w, wsum);
  s_sy[threadIdx.x] = sy;
  s_sq[threadIdx.x] = sq;
  s_lo[threadIdx.x] = lo;
  s_hi[threadIdx.x] = hi;
  __syncthreads();
  // fixed-order tree reduction: deterministic sums
  for (int off = kTT / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      s_sy[threadIdx.x] += s_sy[threadIdx.x + off];
      s_sq[threadIdx.x] += s_sq[threadIdx.x + off];
      s_lo[threadIdx.x] = fminf(s_lo[threadIdx.x], s_lo[threadIdx.x + off]);
      s_hi[threadIdx.x] = fmaxf(s_hi[threadIdx.x], s_hi[threadIdx.x + off]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int slot = nd.slot;
    const unsigned long long nw = s_w;
    bool pure;
    if (pr.crit == SLM_MSE) {
      tr.leaf_value[slot] = nw ? s_sy[0] / (double)nw : 0.0;
      tr.leaf_class[slot] = -1;
      pure = !(s_hi[0] > s_lo[0]);
      par[2 * l] = s_sy[0];
      par[2 * l + 1] = s_sq[0];
    } else {
      int best = 0, nonzero = 0;
      for (int k = 0; k < K; ++k) {
        const unsigned long long c = s_cnt[k];
        cls[(int64_t)l * K + k] = (uint32_t)c;
        if (c > s_cnt[best]) best = k;
        nonzero += c > 0;
      }
      tr.leaf_class[slot] = best;
      tr.leaf_value[slot] = 0.0;
      pure = nonzero <= 1;
    }
    tr.kind[slot] = 0;
    tr.weight[slot] = (int64_t)nw;
    tr.bin[slot] = -1;
    splittable[l] = (nd.depth < max_depth) &&
                    nw >= 2ull * (unsigned long long)pr.min_leaf && !pure;
  }
}

__global__ void __launch_bounds__(kTT)
    k_partition(Problem pr, Swarm sw, const NodeDesc* __restrict__ snodes,
                const int32_t* __restrict__ map, const uint32_t* cls,
                const double* par, TreeArrays tr, uint8_t* side, int32_t* out3,
                int32_t* status) {
  const int a = blockIdx.x;
  const NodeDesc nd = snodes[a];
  const EvalRes gb = sw.gb[a];
  extern __shared__ float s_g[];  // [d]
  __shared__ unsigned long long s_lk[kMaxClasses];
  __shared__ unsigned long long s_wl;
  __shared__ int s_cnt[kTT / 32 + 1];
  const int d = pr.d, K = pr.K;
  if (!gb.valid) {
    if (threadIdx.x == 0) {
      out3[3 * a] = 0;
      out3[3 * a + 1] = 0;
      out3[3 * a + 2] = 0;
    }
    return;
  }
  for (int j = threadIdx.x; j < d; j += kTT) s_g[j] = sw.gbest[(int64_t)a * d + j];
  if (threadIdx.x < kMaxClasses) s_lk[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_wl = 0;
  __syncthreads();
  int n_left_entries = 0;
  unsigned long long wl = 0;
  for (int r = threadIdx.x; r < nd.seg_len; r += kTT) {
    const int64_t e = (int64_t)nd.seg_start + r;
    const float z = project_row(pr.X + e * d, s_g, d);
    const int b = bin_of(z, gb.zmin, gb.inv_w, pr.B);
    const int right = b >= gb.bin;
    side[e] = (uint8_t)right;
    if (!right) {
      const uint32_t w = pr.w ? pr.w[e] : 1u;
      ++n_left_entries;
      wl += w;
      if (pr.crit != SLM_MSE) atomicAdd(&s_lk[pr.lab[e]], (unsigned long long)w);
    }
  }
  atomicAdd(&s_wl, wl);
  int total_left;
  block_excl_scan(n_left_entries, &total_left, s_cnt);
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int l = map[a];
  const int slot = nd.slot;
  const unsigned long long wleft = s_wl;
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
      if (s_lk[k] * nw != (unsigned long long)cls[(int64_t)l * K + k] * wleft)
        no_gain = false;
  }
  out3[3 * a] = no_gain ? 0 : 1;
  out3[3 * a + 1] = total_left;
  out3[3 * a + 2] = nd.seg_len - total_left;
  if (no_gain) return;
  tr.kind[slot] = 1;
  for (int j = 0; j < d; ++j) tr.dir[(int64_t)slot * d + j] = s_g[j];
  tr.zmin[slot] = gb.zmin;
  tr.inv_w[slot] = gb.inv_w;
  tr.bin[slot] = gb.bin;
  tr.loss[slot] = gb.loss;
  tr.n_left[slot] = gb.nl;
  tr.n_right[slot] = gb.nr;
}

__global__ void __launch_bounds__(kTT)
    k_compact(Problem pr, const NodeDesc* __restrict__ snodes,
              const uint8_t* __restrict__ side, const int32_t* __restrict__ dst,
              const int32_t* __restrict__ idx_cur, LevelArrays nx) {
  const int a = blockIdx.x;
  const int dl = dst[2 * a], dr = dst[2 * a + 1];
  if (dl < 0) return;
  const NodeDesc nd = snodes[a];
  const int d = pr.d;
  __shared__ int sbuf[kTT / 32 + 1];
  __shared__ int s_dst[kTT];
  int base_l = 0, base_r = 0;
  for (int t0 = 0; t0 < nd.seg_len; t0 += kTT) {
    const int r = t0 + threadIdx.x;
    const bool in = r < nd.seg_len;
    const int64_t e = (int64_t)nd.seg_start + r;
    const int right = in ? side[e] : 0;
    const int is_left = in && !right;
    int tot_l;
    const int rank_l = block_excl_scan(is_left, &tot_l, sbuf);
    const int n_in = min(kTT, nd.seg_len - t0);
    const int rank_r = threadIdx.x - rank_l;  // entries before r that went right
    if (in) {
      const int32_t pos = is_left ? dl + base_l + rank_l : dr + base_r + rank_r;
      s_dst[threadIdx.x] = pos;
      nx.idx[pos] = idx_cur[e];
      if (nx.lab) nx.lab[pos] = pr.lab[e];
      if (nx.y) nx.y[pos] = pr.y[e];
      if (nx.w) nx.w[pos] = pr.w[e];
    }
    __syncthreads();
    // rows: coalesced copies, one row per group of threads
    for (int q = threadIdx.x; q < n_in * d; q += kTT) {
      const int rr = q / d, j = q - rr * d;
      nx.X[(int64_t)s_dst[rr] * d + j] = pr.X[((int64_t)nd.seg_start + t0 + rr) * d + j];
    }
    __syncthreads();
    base_l += tot_l;
    base_r += n_in - tot_l;
  }
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

__global__ void __launch_bounds__(kTT)
    k_compact_nonzero(const uint32_t* __restrict__ w_all, int64_t n,
                      int32_t* idx_out, uint32_t* w_out,
                      const int64_t* __restrict__ off, int32_t* counts) {
  const int t = blockIdx.x;
  const uint32_t* w = w_all + (int64_t)t * n;
  __shared__ int sbuf[kTT / 32 + 1];
  int64_t base = off[t];
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

__global__ void k_iota(int32_t* idx, int64_t n, int copies) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * copies) idx[i] = (int32_t)(i % n);
}

__global__ void k_validate(const int32_t* labels, int64_t n, int K,
                           const int32_t* idx, int64_t n_idx, int32_t* status) {
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

__global__ void k_predict(const float* __restrict__ X, int64_t n, int d,
                          TreeArrays tr, int n_trees, int H, int B, int K,
                          int crit, int32_t* class_out, double* value_out,
                          int32_t* leaf_out) {
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

}  // namespace

cudaError_t launch_node_stats(const Problem& pr, const LevelNode* nodes, int L,
                              TreeArrays tr, int max_depth, uint32_t* cls,
                              double* par, int32_t* splittable,
                              cudaStream_t st) {
  if (L <= 0) return cudaSuccess;
  k_node_stats<<<L, kTT, 0, st>>>(pr, nodes, tr, max_depth, cls, par,
                                  splittable);
  return cudaGetLastError();
}

cudaError_t launch_partition(const Problem& pr, const Swarm& sw,
                             const NodeDesc* snodes, const int32_t* map, int A,
                             const uint32_t* cls, const double* par,
                             TreeArrays tr, uint8_t* side, int32_t* out3,
                             int32_t* status, cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  k_partition<<<A, kTT, sizeof(float) * pr.d, st>>>(pr, sw, snodes, map, cls,
                                                     par, tr, side, out3,
                                                     status);
  return cudaGetLastError();
}

cudaError_t launch_compact(const Problem& pr, const NodeDesc* snodes, int A,
                           const uint8_t* side, const int32_t* dst,
                           const int32_t* idx_cur, LevelArrays next,
                           cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  k_compact<<<A, kTT, 0, st>>>(pr, snodes, side, dst, idx_cur, next);
  return cudaGetLastError();
}

cudaError_t launch_gather(const float* X, const int32_t* labels, const float* y,
                          const int32_t* idx, int64_t E, int d, float* Xl,
                          int32_t* lab_l, float* y_l, cudaStream_t st) {
  const int64_t total = E * d;
  if (total <= 0) return cudaSuccess;
  k_gather<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(X, labels, y, idx, E, d, Xl,
                                                           lab_l, y_l);
  return cudaGetLastError();
}

cudaError_t launch_compact_nonzero(const uint32_t* w_all, int n_trees,
                                   int64_t n, int32_t* idx_out,
                                   uint32_t* w_out, const int64_t* off,
                                   int32_t* counts, cudaStream_t st) {
  if (n_trees <= 0) return cudaSuccess;
  k_compact_nonzero<<<n_trees, kTT, 0, st>>>(w_all, n, idx_out, w_out, off,
                                             counts);
  return cudaGetLastError();
}

cudaError_t launch_iota(int32_t* idx, int64_t n, int copies, cudaStream_t st) {
  const int64_t total = n * copies;
  if (total <= 0) return cudaSuccess;
  k_iota<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(idx, n, copies);
  return cudaGetLastError();
}

cudaError_t launch_validate(const int32_t* labels, int64_t n, int K,
                            const int32_t* idx, int64_t n_idx,
                            int32_t* status, cudaStream_t st) {
  const int64_t m = (labels && n > n_idx) ? n : n_idx;
  if (m <= 0) return cudaSuccess;
  k_validate<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(labels, n, K, idx,
                                                          n_idx, status);
  return cudaGetLastError();
}

cudaError_t launch_predict(const float* X, int64_t n, int d, TreeArrays tr,
                           int n_trees, int H, int B, int K, int crit,
                           int32_t* class_out, double* value_out,
                           int32_t* leaf_out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_predict<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
      X, n, d, tr, n_trees, H, B, K, crit, class_out, value_out, leaf_out);
  return cudaGetLastError();
}

}  // namespace slm
