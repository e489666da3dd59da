// Probabilistic search of the original SLM (Sec. II-B, Eqs. dynamic and
// exp_a): the projection search that the swarm search replaces, kept as a
// GPU baseline. The node's features are ranked by their own split loss;
// every candidate vector picks R of the D ranks (rank r with weight
// gamma^(r-1), without replacement) and gives each an integer coefficient in
// [-m_r, m_r], m_r = floor(alpha0 exp(-alpha r)); candidates are scored in
// batches by the split-scoring kernels and the best is kept (strictly
// better replaces: ties to the lower candidate). A cosine pruning then keeps
// a diverse set of the best candidates (exact integer test).
#include <cuda_runtime.h>
#include <limits.h>

#include <algorithm>

#include "device_util.cuh"
#include "philox.cuh"
#include "slm_internal.cuh"

namespace slm {
namespace {

constexpr uint32_t kProbPurpose = 9;

// Candidates c0 .. c0 + count - 1, one thread each: row i of pos[Pp, d]
// (rows count .. Pp - 1 zero) and row c0 + i of all_pos[I, d]. w[r]: the
// selection weight of rank r + 1 (gamma^r); m[r]: its coefficient range.
// Draw k is lane k mod 4 of Philox(seed, {uid, c, k / 4, 9 << 24}).
__global__ void k_prob_candidates(uint64_t seed, uint32_t uid, int c0, int count, int Pp, int d,
                                  const int32_t* __restrict__ rank_feat,
                                  const double* __restrict__ w, const int32_t* __restrict__ m,
                                  int R, float* __restrict__ pos, float* __restrict__ all_pos) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Pp) return;
  float* row = pos + (int64_t)i * d;
  for (int j = 0; j < d; ++j) row[j] = 0.0f;
  if (i >= count) return;
  const uint32_t c = (uint32_t)(c0 + i);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  uint32_t used[kMaxD / 32];
  for (int q = 0; q < (d + 31) / 32; ++q) used[q] = 0u;
  int chosen[kProbMaxR];
  U4 r4{};
  for (int k = 0; k < 2 * R; ++k) {
    if ((k & 3) == 0) r4 = philox4x32_10(uid, c, (uint32_t)(k >> 2), kProbPurpose << 24, k0, k1);
    const double u = (double)uniform24(r4.v[k & 3]);
    if (k < R) {
      double total = 0.0;
      for (int r = 0; r < d; ++r)
        if (!((used[r >> 5] >> (r & 31)) & 1u)) total = __dadd_rn(total, w[r]);
      const double target = __dmul_rn(u, total);
      double run = 0.0;
      int pick = -1, last = -1;
      for (int r = 0; r < d; ++r) {
        if ((used[r >> 5] >> (r & 31)) & 1u) continue;
        last = r;
        run = __dadd_rn(run, w[r]);
        if (run > target) {
          pick = r;
          break;
        }
      }
      if (pick < 0) pick = last;
      used[pick >> 5] |= 1u << (pick & 31);
      chosen[k] = pick;
    } else {
      const int r = chosen[k - R];
      const double mr = (double)m[r];
      row[rank_feat[r]] = (float)(floor(__dmul_rn(u, __dadd_rn(__dmul_rn(2.0, mr), 1.0))) - mr);
    }
  }
  float* arow = all_pos + (int64_t)c * d;
  for (int j = 0; j < d; ++j) arow[j] = row[j];
}

// After the batch of candidates c0 .. c0 + P - 1 (pr.P = its size) was
// scored into cur[]: the best so far is replaced by the batch's best if
// strictly better (gbest_argmin with gold = the best so far; at b = 0 every
// candidate qualifies), its vector copied, trace[b] and all_scores updated.
__global__ void k_prob_best(Problem pr, const EvalRes* __restrict__ cur, int c0, int b,
                            EvalRes* best, int32_t* best_idx, const float* __restrict__ all_pos,
                            float* best_pos, double* trace, EvalRes* all_scores) {
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < pr.P; i += blockDim.x) all_scores[c0 + i] = cur[i];
  if (threadIdx.x >= 32) return;
  const EvalRes gold = *best;
  EvalRes be;
  const int bi = gbest_argmin(pr, cur, gold, b, &be);
  const int32_t idx = bi >= 0 ? c0 + bi : *best_idx;
  if (bi >= 0) {
    for (int j = lane; j < pr.d; j += 32) best_pos[j] = all_pos[(int64_t)idx * pr.d + j];
  }
  if (lane == 0) {
    const EvalRes g = bi >= 0 ? be : gold;
    if (bi >= 0) {
      *best = be;
      *best_idx = idx;
    }
    if (trace) trace[b] = g.valid ? g.loss : __longlong_as_double(0x7ff0000000000000LL);
  }
}

// Unit vectors e_{c0} .. e_{c0 + count - 1} as rows of pos[Pp, d] (the
// feature ranking scores each feature alone); rows count .. Pp - 1 zero.
__global__ void k_prob_units(int c0, int count, int Pp, int d, float* __restrict__ pos) {
  const int64_t total = (int64_t)Pp * d;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(k / d), j = (int)(k % d);
    pos[k] = (i < count && j == c0 + i) ? 1.0f : 0.0f;
  }
}

__global__ void k_prob_init(EvalRes* best, int32_t* best_idx) {
  *best = invalid_res();
  *best_idx = 0;
}

// Cosine pruning by one CTA: q times, the best candidate not yet pruned and
// not the zero vector is kept (exact score order, ties to the lower index),
// then every live candidate with cos_den^2 dot^2 > cos_num^2 |a|^2 |b|^2 to
// it (itself included) is pruned. pruned[I] is scratch.
__global__ void __launch_bounds__(256)
    k_prob_prune(int crit, int I, int d, const float* __restrict__ all_pos,
                 const EvalRes* __restrict__ sc, int q, int64_t cn2, int64_t cd2,
                 uint8_t* pruned, int32_t* kept, int32_t* n_kept) {
  __shared__ int s_idx[8];
  __shared__ int s_pick;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = threadIdx.x; c < I; c += blockDim.x) {
    int64_t nrm = 0;
    for (int j = 0; j < d; ++j) {
      const int64_t v = (int64_t)all_pos[(int64_t)c * d + j];
      nrm += v * v;
    }
    pruned[c] = nrm == 0;
  }
  __syncthreads();
  int nk = 0;
  for (; nk < q; ++nk) {
    // best live candidate: per thread, then warp, then block (exact order)
    int bi = -1;
    for (int c = threadIdx.x; c < I; c += blockDim.x)
      if (!pruned[c] && (bi < 0 || better(sc[c], sc[bi], crit))) bi = c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (oi >= 0 && (bi < 0 || better(sc[oi], sc[bi], crit) ||
                      (!better(sc[bi], sc[oi], crit) && oi < bi)))
        bi = oi;
    }
    if (lane == 0) s_idx[warp] = bi;
    __syncthreads();
    if (threadIdx.x == 0) {
      int b = -1;
      for (int w2 = 0; w2 < 8; ++w2) {
        const int oi = s_idx[w2];
        if (oi >= 0 && (b < 0 || better(sc[oi], sc[b], crit) ||
                        (!better(sc[b], sc[oi], crit) && oi < b)))
          b = oi;
      }
      s_pick = b;
      if (b >= 0) kept[nk] = b;
    }
    __syncthreads();
    const int b = s_pick;
    if (b < 0) break;
    const float* ab = all_pos + (int64_t)b * d;
    int64_t na = 0;
    for (int j = 0; j < d; ++j) na += (int64_t)ab[j] * (int64_t)ab[j];
    for (int c = threadIdx.x; c < I; c += blockDim.x) {
      if (pruned[c]) continue;
      const float* ac = all_pos + (int64_t)c * d;
      int64_t dot = 0, nc = 0;
      for (int j = 0; j < d; ++j) {
        dot += (int64_t)ab[j] * (int64_t)ac[j];
        nc += (int64_t)ac[j] * (int64_t)ac[j];
      }
      if (c == b || cd2 * dot * dot > cn2 * na * nc) pruned[c] = 1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_kept = nk;
}

}  // namespace

cudaError_t launch_prob_init(EvalRes* best, int32_t* best_idx, cudaStream_t st) {
  k_prob_init<<<1, 1, 0, st>>>(best, best_idx);
  return cudaGetLastError();
}

cudaError_t launch_prob_units(int c0, int count, int Pp, int d, float* pos, cudaStream_t st) {
  const int64_t total = (int64_t)Pp * d;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 1024);
  k_prob_units<<<blocks, 256, 0, st>>>(c0, count, Pp, d, pos);
  return cudaGetLastError();
}

cudaError_t launch_prob_candidates(uint64_t seed, uint32_t uid, int c0, int count, int Pp, int d,
                                   const int32_t* rank_feat, const double* w, const int32_t* m,
                                   int R, float* pos, float* all_pos, cudaStream_t st) {
  k_prob_candidates<<<(Pp + 63) / 64, 64, 0, st>>>(seed, uid, c0, count, Pp, d, rank_feat, w, m,
                                                    R, pos, all_pos);
  return cudaGetLastError();
}

cudaError_t launch_prob_best(const Problem& pr, const EvalRes* cur, int c0, int b, EvalRes* best,
                             int32_t* best_idx, const float* all_pos, float* best_pos,
                             double* trace, EvalRes* all_scores, cudaStream_t st) {
  k_prob_best<<<1, 128, 0, st>>>(pr, cur, c0, b, best, best_idx, all_pos, best_pos, trace,
                                 all_scores);
  return cudaGetLastError();
}

cudaError_t launch_prob_prune(int crit, int I, int d, const float* all_pos, const EvalRes* sc,
                              int q, int64_t cos_num, int64_t cos_den, uint8_t* pruned,
                              int32_t* kept, int32_t* n_kept, cudaStream_t st) {
  k_prob_prune<<<1, 256, 0, st>>>(crit, I, d, all_pos, sc, q, cos_num * cos_num,
                                  cos_den * cos_den, pruned, kept, n_kept);
  return cudaGetLastError();
}

}  // namespace slm
