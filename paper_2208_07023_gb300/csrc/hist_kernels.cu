// Histogram and threshold scan of classification searches in the FP32 form
// (Sec. II-A, Eqs. 1, 3-4: bins of the projection, class counts, the
// weighted Gini or entropy of every interior edge; Algorithm 1's pbest step).
//
// One CTA per (node, particle, slice); the S slices of a (node, particle)
// form a cluster. The kernel is a chain of short phases, each built to keep
// its latency off the critical path:
//  * before the previous kernel's results are visible (programmatic
//    dependent launch): the histogram copies are zeroed and, for the pbest
//    rank, the Philox draws of the next move are taken;
//  * binning: every thread keeps 16 entries in flight (four 16-byte loads of
//    z, of labels, of multiplicities) before their shared-memory atomics,
//    into the copy of its warp pair; histograms are class-major ([K][B]);
//  * the copies are summed, and the cluster's ranks sum one slice each of
//    every rank's counters through distributed shared memory into rank 0;
//  * the scan: one warp per class turns the class's row of B bins into its
//    prefix sums (16-byte loads, a shuffle scan), then thread b scores edge
//    b + 1 (bins <= b left) from the K prefixes at bin b (consecutive threads
//    read consecutive words) and the class totals at bin B - 1. The edge
//    rules and arithmetic are those of block_scan_cls
//    (Gini: the exact rational by 128-bit cross-multiplication; entropy:
//    c ln c summed in class order; repeated partitions skipped, ties to the
//    lower edge), so the scores are identical;
//  * the pbest step and the gB-independent move terms are spread over the
//    CTA's threads; in a node-step search (Swarm::node_step) the last CTA to
//    score a node then takes the node's gbest step and moves its particles
//    (one CTA per node instead of every projection CTA), else k_step
//    finishes the move.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <float.h>
#include <limits.h>

#include "device_util.cuh"
#include "philox.cuh"
#include "scan_util.cuh"
#include "slm_internal.cuh"

namespace slm {
namespace {

constexpr int kHcCopies = 4;  // histogram copies, one per pair of warps
constexpr int kHcWarps = kThreads / 32;

struct HcScratch {
  uint64_t wn[kHcWarps], wd[kHcWarps];
  double wl[kHcWarps];
  int wb[kHcWarps];
  uint32_t wnl[kHcWarps];
  EvalRes res;
  EvalRes pb, gb;  // the particle's pbest score and the node's gbest score (prefetched)
  float zmin, inv_w;
  int ok, imp;
};

// Floats of one d-vector in the kernel's shared memory (16-byte multiples).
__host__ __device__ inline int hc_dvec(int d) { return (d + 3) & ~3; }

// Words of the histogram region: the copies, or (reused by the BF16 form's
// top-k selection) P scores and 2 P indices when those need more; a
// multiple of 4.
__host__ __device__ inline int hc_words(int B, int K, int P) {
  const int copies = kHcCopies * B * K;
  const int topk = (int)((sizeof(EvalRes) + 8) * P / 4);
  return ((copies > topk ? copies : topk) + 3) & ~3;
}

// A double's total order as an unsigned key (negative values below 0).
__device__ __forceinline__ uint64_t hc_key(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  return (u >> 63) ? ~u : u | 0x8000000000000000ull;
}

__device__ __forceinline__ double xlogx_tab(const double* tab, uint32_t c) {
  return (tab && c < (uint32_t)kXlogxTab) ? __ldg(tab + c) : xlogx(c);
}

// Edge order of the scan: a better score, ties to the lower edge (bb < 0:
// none). Gini scores are rationals n / d (larger is better), entropy a loss.
template <int CRIT>
__device__ __forceinline__ bool hc_takes(uint64_t on, uint64_t od, double ol, int ob, uint64_t bn,
                                         uint64_t bd, double bl, int bb) {
  if (ob < 0) return false;
  if (bb < 0) return true;
  if (CRIT == SLM_GINI) return prod_gt(on, bd, bn, od) || (!prod_gt(bn, od, on, bd) && ob < bb);
  return ol < bl || (!(bl < ol) && ob < bb);
}

template <int CRIT>
__global__ void __launch_bounds__(kThreads, 2)
    k_hist_cls(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes,
               const int32_t* __restrict__ list, int t, int do_update,
               const double* __restrict__ xtab) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ HcScratch sc;
  const cg::cluster_group cl = cg::this_cluster();
  pdl_trigger();
  const int S = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int a = list ? list[blockIdx.x / S] : (int)blockIdx.x / S;
  const int p = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int B = pr.B, K = pr.K, W = B * K, d = pr.d;
  const NodeDesc nd = nodes[a];
  const int dv = hc_dvec(d);
  uint32_t* hc = reinterpret_cast<uint32_t*>(smem);           // [kHcCopies][W]
  float* c1u = reinterpret_cast<float*>(hc + hc_words(B, K, pr.P));  // [d] c1 r1 of the next move
  float* s2u = c1u + dv;                                      // [d] c2 r2
  float* xrow = s2u + dv;                                     // [d] the particle's x, v, pB
  float* vrow = xrow + dv;
  float* prow = vrow + dv;
  const bool premove = do_update && sw.ic && t < sw.T && rank == 0;

  // work that does not wait for the projection: zero the copies, draw the
  // next move's r1 and r2 (counter (uid, t + 1, p, j / 4), as move_item)
  for (int i = threadIdx.x; i < kHcCopies * W; i += kThreads) hc[i] = 0u;
  if (premove) {
    const uint32_t k0 = (uint32_t)sw.co.seed, k1 = (uint32_t)(sw.co.seed >> 32);
    for (int q = threadIdx.x; q < ((d + 3) >> 2); q += kThreads) {
      const U4 r1 = philox4x32_10(nd.uid, (uint32_t)(t + 1), (uint32_t)p,
                                  (uint32_t)q | (kR1 << 24), k0, k1);
      const U4 r2 = philox4x32_10(nd.uid, (uint32_t)(t + 1), (uint32_t)p,
                                  (uint32_t)q | (kR2 << 24), k0, k1);
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (4 * q + c < d) {
          c1u[4 * q + c] = __fmul_rn(sw.co.c1, uniform24(r1.v[c]));
          s2u[4 * q + c] = __fmul_rn(sw.co.c2, uniform24(r2.v[c]));
        }
    }
  }
  __syncthreads();  // the zeroed copies, before any binning
  pdl_wait();
  int* zz = sw.zmm + ((int64_t)a * pr.Pp + p) * 2;
  const int64_t ci = (int64_t)a * pr.Pp + p;
  // this rank's slice (starts on a multiple of 4 entries)
  const int chunk = ((nd.seg_len + S - 1) / S + 3) & ~3;
  const int r_begin = min(nd.seg_len, rank * chunk);
  const int r_end = min(nd.seg_len, r_begin + chunk);
  const int64_t e0 = nd.seg_start + r_begin;
  const float* zs = sw.z + (int64_t)p * pr.Ez + e0;
  const int32_t* ls = pr.lab + e0;
  const uint32_t* ws = pr.w ? pr.w + e0 : nullptr;
  const int n = r_end - r_begin;
  const bool g16 = (e0 & 3) == 0;  // 16-byte loads: groups of four entries
  const int n4 = g16 ? n >> 2 : 0;
  constexpr int U = 4;  // groups in flight per thread
  float4 zv[U];
  int4 lv[U];
  uint4 wv[U];
  auto load_groups = [&](int g0) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int g = g0 + u * kThreads;
      const bool in = g < n4;
      zv[u] = in ? __ldcg(reinterpret_cast<const float4*>(zs) + g) : make_float4(0, 0, 0, 0);
      lv[u] = in ? __ldg(reinterpret_cast<const int4*>(ls) + g) : make_int4(-1, -1, -1, -1);
      wv[u] = in && ws ? __ldg(reinterpret_cast<const uint4*>(ws) + g) : make_uint4(1, 1, 1, 1);
    }
  };
  // the first groups are in flight while the range is read
  load_groups(threadIdx.x);
  // the tail's inputs, also in flight from here: the particle's pbest score
  // and the node's gbest score (evaluation t - 1), its x, v and pB rows
  const int64_t prow0 = ci * d;
  if (do_update && rank == 0) {
    constexpr int kResWords = (int)(sizeof(EvalRes) / 4);
    const int64_t gi = (int64_t)((t + 1) & 1) * sw.n_nodes + a;
    if (threadIdx.x < kResWords)
      cp_async4(reinterpret_cast<uint32_t*>(&sc.pb) + threadIdx.x,
                reinterpret_cast<const uint32_t*>(sw.pb + ci) + threadIdx.x, 4);
    else if (threadIdx.x >= 32 && threadIdx.x < 32 + kResWords && sw.imp)
      cp_async4(reinterpret_cast<uint32_t*>(&sc.gb) + (threadIdx.x - 32),
                reinterpret_cast<const uint32_t*>(sw.gb + gi) + (threadIdx.x - 32), 4);
    for (int j = threadIdx.x; j < d; j += kThreads) {
      cp_async4(xrow + j, sw.pos + prow0 + j, 4);
      if (premove) {
        cp_async4(vrow + j, sw.vel + prow0 + j, 4);
        cp_async4(prow + j, sw.pbest + prow0 + j, 4);
      }
    }
    cp_async_commit();
  }
  // the particle's range, read and turned into the bin width by every
  // thread (the same values everywhere; thread 0 resets the range only
  // after the barriers below)
  float zmin = 0.f, inv_w = 0.f;
  bool ok = false;
  {
    const int lo_o = __ldcg(zz), hi_o = __ldcg(zz + 1);
    if (lo_o != INT_MAX) {
      const float lo = ord2f(lo_o), hi = ord2f(hi_o);
      inv_w = __fdiv_rn((float)B, __fsub_rn(hi, lo));
      zmin = lo;
      ok = (hi > lo) && isfinite(inv_w);
    }
  }

  // ---- binning of this rank's slice
  if (ok) {
    uint32_t* h = hc + (warp % kHcCopies) * W;  // class-major: h[label * B + bin]
    int done = 0;
    if (g16) {
      for (int g0 = threadIdx.x; g0 < n4; g0 += U * kThreads) {
        if (g0 != (int)threadIdx.x) load_groups(g0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (lv[u].x < 0) continue;  // past the slice (whole group)
          atomicAdd(&h[lv[u].x * B + bin_of(zv[u].x, zmin, inv_w, B)], wv[u].x);
          atomicAdd(&h[lv[u].y * B + bin_of(zv[u].y, zmin, inv_w, B)], wv[u].y);
          atomicAdd(&h[lv[u].z * B + bin_of(zv[u].z, zmin, inv_w, B)], wv[u].z);
          atomicAdd(&h[lv[u].w * B + bin_of(zv[u].w, zmin, inv_w, B)], wv[u].w);
        }
      }
      done = n4 << 2;
    }
    for (int i = done + (int)threadIdx.x; i < n; i += kThreads) {
      const int b = bin_of(__ldcg(zs + i), zmin, inv_w, B);
      atomicAdd(&h[__ldg(ls + i) * B + b], ws ? __ldg(ws + i) : 1u);
    }
  }
  __syncthreads();
  // ---- the copies into copy 0
  for (int i = threadIdx.x; i < W; i += kThreads) {
    uint32_t v = hc[i];
#pragma unroll
    for (int c = 1; c < kHcCopies; ++c) v += hc[c * W + i];
    hc[i] = v;
  }
  // ---- the cluster's histograms into rank 0: rank r sums the r-th of S
  // slices of the counters over every rank (all loads in flight at once)
  // and stores the sums into rank 0's copy (the slices are disjoint)
  if (S > 1) {
    cl.sync();  // every rank's copy 0 is complete
    const int per = (W + S - 1) / S;
    const int lo = rank * per, hi = min(W, lo + per);
    uint32_t* h0 = cl.map_shared_rank(hc, 0);
    for (int i = lo + (int)threadIdx.x; i < hi; i += kThreads) {
      uint32_t v = 0;
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (q < S) v += cl.map_shared_rank(hc, q)[i];
      h0[i] = v;
    }
    cl.sync();  // rank 0's counters are complete; no rank reads another's
    if (rank != 0) return;
  }
  cp_async_wait<0>();  // the tail's prefetched inputs
  __syncthreads();

  // ---- threshold scan
  EvalRes res = invalid_res();
  if (ok) {
    // 1. each class's row of bins into inclusive prefix sums, in place:
    //    warp w takes classes w, w + 8, ...; lane l holds bins l*bpl ..
    const int bpl = (B + 31) >> 5;
    const bool vec4 = B == 32 * bpl && (bpl & 3) == 0;  // rows of 4-bin words
    // two classes per warp at a time (k and k + 8), their scans interleaved
    auto load_row = [&](const uint32_t* row, uint32_t* v) {
      if (vec4) {
#pragma unroll
        for (int i = 0; i < 8; i += 4)
          if (i < bpl) {
            const uint4 q = *reinterpret_cast<const uint4*>(row + lane * bpl + i);
            v[i] = q.x;
            v[i + 1] = q.y;
            v[i + 2] = q.z;
            v[i + 3] = q.w;
          }
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int j = lane * bpl + i;
          v[i] = (i < bpl && j < B) ? row[j] : 0u;
        }
      }
    };
    auto store_row = [&](uint32_t* row, const uint32_t* v) {
      if (vec4) {
#pragma unroll
        for (int i = 0; i < 8; i += 4)
          if (i < bpl)
            *reinterpret_cast<uint4*>(row + lane * bpl + i) =
                make_uint4(v[i], v[i + 1], v[i + 2], v[i + 3]);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int j = lane * bpl + i;
          if (i < bpl && j < B) row[j] = v[i];
        }
      }
    };
    for (int k0 = warp; k0 < K; k0 += 2 * kHcWarps) {
      const int k1 = k0 + kHcWarps;
      const bool two = k1 < K;
      uint32_t v0[8] = {}, v1[8] = {};
      load_row(hc + k0 * B, v0);
      if (two) load_row(hc + k1 * B, v1);
      uint32_t s0 = 0, s1 = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < bpl) {
          s0 += v0[i];
          s1 += v1[i];
        }
      uint32_t in0 = s0, in1 = s1;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t u0 = __shfl_up_sync(0xffffffffu, in0, off);
        const uint32_t u1 = __shfl_up_sync(0xffffffffu, in1, off);
        if (lane >= off) {
          in0 += u0;
          in1 += u1;
        }
      }
      uint32_t r0 = in0 - s0, r1 = in1 - s1;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < bpl) {
          r0 += v0[i];
          v0[i] = r0;
          r1 += v1[i];
          v1[i] = r1;
        }
      store_row(hc + k0 * B, v0);
      if (two) store_row(hc + k1 * B, v1);
    }
    __syncthreads();
    // 2. thread b scores edge e = b + 1 (bins <= b left); an empty bin b
    //    repeats edge b's split and is skipped
    const int b = threadIdx.x;
    uint64_t bn = 0, bd = 0;
    double bl = 0.0;
    int bb = -1;
    uint32_t bnl = 0, ntot = 0;
    if (b <= B - 2) {
      uint32_t nl = 0, prev = 0;
      uint64_t sl = 0, sr = 0;
      double hl = 0.0, hr = 0.0;
#pragma unroll 4
      for (int k = 0; k < K; ++k) {
        const uint32_t* row = hc + k * B;
        const uint32_t l = row[b], tk = row[B - 1], r = tk - l;
        nl += l;
        ntot += tk;
        if (b > 0) prev += row[b - 1];
        if (CRIT == SLM_GINI) {
          sl += (uint64_t)l * l;
          sr += (uint64_t)r * r;
        } else {
          hl += xlogx_tab(xtab, l);
          hr += xlogx_tab(xtab, r);
        }
      }
      const uint32_t nr = ntot - nl;
      if (nl != prev && nl >= (uint32_t)pr.min_leaf && nr >= (uint32_t)pr.min_leaf) {
        bb = b + 1;
        bnl = nl;
        if (CRIT == SLM_GINI) {
          bn = sl * nr + sr * nl;
          bd = (uint64_t)nl * nr;
        } else {
          bl = ((xlogx_tab(xtab, nl) - hl) + (xlogx_tab(xtab, nr) - hr)) / (double)ntot;
        }
      }
    }
    // block argmin over the edges (ties to the lower edge), on a key of the
    // loss each edge would report (Gini: (n d - q) / (n d) from the exact
    // rational, in float, so no double division per edge; entropy: the
    // double loss), with edges within 8 ulps of the key's smallest compared
    // exactly in edge order: the key's rounding is far below 8 ulps, so the
    // choice is the exact one
    auto edge_key = [&](uint64_t n_, uint64_t d_, double l_, int b_) -> uint64_t {
      if (b_ < 0) return ~0ull;
      if (CRIT == SLM_GINI) {
        const uint64_t nden = (uint64_t)ntot * d_;
        return __float_as_uint(__fdiv_rn((float)(nden - n_), (float)nden));  // >= 0
      }
      return hc_key(l_);
    };
    uint64_t key = edge_key(bn, bd, bl, bb);
    // the exact winner among this warp's lanes in `cand` (lane order =
    // edge order), into lane 0's bn, bd, bl, bb, bnl
    auto resolve = [&](unsigned cand) {
      int wi = cand ? __ffs(cand) - 1 : 0;
      uint64_t wn = __shfl_sync(0xffffffffu, bn, wi), wd = __shfl_sync(0xffffffffu, bd, wi);
      double wl = __shfl_sync(0xffffffffu, bl, wi);
      int wb = cand ? __shfl_sync(0xffffffffu, bb, wi) : -1;
      uint32_t wnl = __shfl_sync(0xffffffffu, bnl, wi);
      unsigned m = cand ? cand & (cand - 1) : 0u;
      while (m) {  // rare: several edges within a few ulps
        const int li = __ffs(m) - 1;
        m &= m - 1;
        const uint64_t on = __shfl_sync(0xffffffffu, bn, li), od = __shfl_sync(0xffffffffu, bd, li);
        const double ol = __shfl_sync(0xffffffffu, bl, li);
        const int ob = __shfl_sync(0xffffffffu, bb, li);
        const uint32_t onl = __shfl_sync(0xffffffffu, bnl, li);
        if (hc_takes<CRIT>(on, od, ol, ob, wn, wd, wl, wb)) {
          wn = on;
          wd = od;
          wl = ol;
          wb = ob;
          wnl = onl;
        }
      }
      bn = wn;
      bd = wd;
      bl = wl;
      bb = wb;
      bnl = wnl;
    };
    {
      uint64_t kmin;
      if (CRIT == SLM_GINI) {  // a 32-bit key: one reduction
        kmin = __reduce_min_sync(0xffffffffu, bb >= 0 ? (uint32_t)key : 0xffffffffu);
      } else {
        kmin = key;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const uint64_t o = __shfl_xor_sync(0xffffffffu, kmin, off);
          kmin = o < kmin ? o : kmin;
        }
      }
      resolve(__ballot_sync(0xffffffffu, bb >= 0 && key <= kmin + 8));
    }
    if (lane == 0) {
      sc.wn[warp] = bn;
      sc.wd[warp] = bd;
      sc.wl[warp] = bl;
      sc.wb[warp] = bb;
      sc.wnl[warp] = bnl;
    }
    __syncthreads();
    if (warp == 0) {
      const bool in = lane < kHcWarps;
      const uint32_t nt = ntot;  // every edge's thread summed the class totals
      bn = in ? sc.wn[lane] : 0;
      bd = in ? sc.wd[lane] : 0;
      bl = in ? sc.wl[lane] : 0.0;
      bb = in ? sc.wb[lane] : -1;
      bnl = in ? sc.wnl[lane] : 0u;
      key = edge_key(bn, bd, bl, bb);
      uint64_t kmin;
      if (CRIT == SLM_GINI) {
        kmin = __reduce_min_sync(0xffffffffu, bb >= 0 ? (uint32_t)key : 0xffffffffu);
      } else {
        kmin = key;
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
          const uint64_t o = __shfl_xor_sync(0xffffffffu, kmin, off);
          kmin = o < kmin ? o : kmin;
        }
      }
      resolve(__ballot_sync(0xffffffffu, bb >= 0 && key <= kmin + 8));
      if (lane == 0 && bb >= 0) {
        res.valid = 1;
        res.bin = bb;
        res.nl = bnl;
        res.nr = nt - bnl;
        if (CRIT == SLM_GINI) {
          res.num = bn;
          res.den = bd;
          const uint64_t nden = (uint64_t)nt * bd;
          res.loss = (double)(nden - bn) / (double)nden;
        } else {
          res.loss = bl;
        }
      }
    }
    if (threadIdx.x == 0) {
      res.zmin = zmin;
      res.inv_w = inv_w;
    }
  }

  // ---- score, range reset, pbest step, the next move's gB-independent terms
  if (threadIdx.x == 0) {
    sw.cur[ci] = res;
    zz[0] = INT_MAX;  // ready for the next iteration
    zz[1] = INT_MIN;
    int imp = 0;
    if (do_update) {
      // mark_improvement's rule on the prefetched gbest score
      if (sw.imp && res.valid && (t == 0 || better(res, sc.gb, pr.crit)))
        atomicOr(sw.imp + (int64_t)(t & 1) * sw.n_nodes + a, 1);
      imp = (t == 0) || better(res, sc.pb, pr.crit);
      if (imp) sw.pb[ci] = res;
    }
    sc.imp = imp;
  }
  if (sw.tk_sel) {
    // the reduced pass of the BF16 form: the last CTA of the node to score
    // its particle selects the node's top k (the histogram copies are free)
    __threadfence();  // this CTA's score write before the count
    __syncthreads();
    if (threadIdx.x == 0) sc.ok = atomicAdd(&sw.done[a], 1) + 1 == pr.P;
    __syncthreads();
    if (sc.ok) {
      __threadfence();
      topk_select(pr, sw, a, reinterpret_cast<unsigned char*>(hc));
      if (threadIdx.x == 0) sw.done[a] = 0;
    }
  }
  if (!do_update) return;
  __syncthreads();
  const bool imp = sc.imp;
  const int64_t row = prow0;
  if (imp || premove)
    for (int j = threadIdx.x; j < d; j += kThreads) {
      const float x = xrow[j];
      if (imp) sw.pbest[row + j] = x;  // the position is kept on improvement
      if (premove) {
        // ic = omega v + (c1 r1)(pB - x); pB is x itself after an improvement
        const float pbv = imp ? x : prow[j];
        sw.ic[row + j] = __fadd_rn(__fmul_rn(sw.co.inertia, vrow[j]),
                                   __fmul_rn(c1u[j], __fsub_rn(pbv, x)));
        sw.s2[row + j] = s2u[j];
      }
    }
  if (!sw.node_step) return;

  // ---- the last particle of the node to be scored: the node's gbest step
  // and (t < T) the move of its particles
  __syncthreads();  // this CTA's score, pbest and move terms are written
  if (threadIdx.x == 0) {
    __threadfence();
    sc.ok = atomicAdd(&sw.done[a], 1) == pr.P - 1;
  }
  __syncthreads();
  if (!sc.ok) return;
  __threadfence();
  const int A = sw.n_nodes, Pn = pr.P;
  const int64_t nb = (int64_t)a * pr.Pp * d;
  const bool move = t < sw.T;
  const bool v4 = (d & 3) == 0;
  const int d4 = d >> 2, items = move && v4 ? Pn * d4 : 0;
  // The positions and the recorded gB go to shared memory (the histograms
  // are done with) by asynchronous copies, the first move terms to
  // registers, all while warp 0 takes the gbest step: after a gbest change
  // gB is the new best particle's position (it beat every pbest, so its own
  // pbest became that position), so the move needs nothing more from memory.
  float* xsm = reinterpret_cast<float*>(hc);
  const bool in_smem = items > 0 && (Pn + 1) * d <= kHcCopies * W;
  if (in_smem) {
    for (int e = threadIdx.x; e < items; e += kThreads)
      cp_async16(xsm + 4 * e, sw.pos + nb + 4 * (int64_t)e, 16);
    for (int q = threadIdx.x; q < d4; q += kThreads)
      cp_async16(xsm + Pn * d + 4 * q, sw.gbest + (int64_t)a * d + 4 * q, 16);
    cp_async_commit();
  }
  constexpr int kNsItems = 4;  // move items per thread in flight
  float4 ia[kNsItems], sa[kNsItems];
  auto load_batch = [&](int e0) {
#pragma unroll
    for (int u = 0; u < kNsItems; ++u) {
      const int e = e0 + u * kThreads;
      if (e < items) {
        const int64_t o = nb + 4 * (int64_t)e;  // item e: features 4 (e mod d4) .. of particle e / d4
        ia[u] = __ldcg(reinterpret_cast<const float4*>(sw.ic + o));
        sa[u] = __ldcg(reinterpret_cast<const float4*>(sw.s2 + o));
      }
    }
  };
  load_batch(threadIdx.x);
  __shared__ int s_best;
  if (warp == 0) {
    // the argmin only when a particle beat gB in this evaluation (every
    // particle is a candidate at evaluation 0)
    const int64_t fi = (int64_t)(t & 1) * A + a;
    const bool any = t == 0 || __ldcg(sw.imp + fi) != 0;
    const EvalRes gold = ldcg_res(sw.gb + (int64_t)((t + 1) & 1) * A + a);
    EvalRes be = gold;
    const int bi = any ? gbest_argmin(pr, sw.cur + (int64_t)a * pr.Pp, gold, t, &be, true) : -1;
    if (lane == 0) {
      sw.imp[fi] = 0;  // ready for evaluation t + 2
      const EvalRes g = bi >= 0 ? be : gold;
      sw.gb[(int64_t)(t & 1) * A + a] = g;
      if (bi >= 0) {
        sw.gpart[a] = bi;
        sw.giter[a] = t;
      }
      if (sw.trace)
        sw.trace[(int64_t)a * (sw.T + 1) + t] =
            g.valid ? g.loss : __longlong_as_double(0x7ff0000000000000LL);
      s_best = bi;
      sw.done[a] = 0;  // ready for the next evaluation
    }
  }
  if (in_smem) cp_async_wait<0>();
  __syncthreads();
  const int bi = s_best;
  // a new best improved its pbest in this evaluation: gB is that row
  const float* gsrc = bi >= 0 ? sw.pbest + nb + (int64_t)bi * d : sw.gbest + (int64_t)a * d;
  const float* gsm = bi >= 0 ? xsm + bi * d : xsm + Pn * d;
  if (bi >= 0)
    for (int j = threadIdx.x; j < d; j += kThreads)
      sw.gbest[(int64_t)a * d + j] = in_smem ? gsm[j] : __ldcg(gsrc + j);
  if (!move) return;
  // x' = x + (ic + s2 (gB - x)), v' = ic + s2 (gB - x), one rounding each
  if (v4) {
    for (int e0 = threadIdx.x; e0 < items; e0 += kNsItems * kThreads) {
      if (e0 != (int)threadIdx.x) load_batch(e0);
#pragma unroll
      for (int u = 0; u < kNsItems; ++u) {
        const int e = e0 + u * kThreads;
        if (e >= items) break;
        const int j = 4 * (e % d4);
        const float4 x = in_smem ? *reinterpret_cast<const float4*>(xsm + 4 * e)
                                 : __ldcg(reinterpret_cast<const float4*>(sw.pos + nb) + e);
        const float4 g = in_smem ? *reinterpret_cast<const float4*>(gsm + j)
                                 : __ldcg(reinterpret_cast<const float4*>(gsrc + j));
        const float4 ic = ia[u], s2 = sa[u];
        float4 vn, xn;
        vn.x = __fadd_rn(ic.x, __fmul_rn(s2.x, __fsub_rn(g.x, x.x)));
        vn.y = __fadd_rn(ic.y, __fmul_rn(s2.y, __fsub_rn(g.y, x.y)));
        vn.z = __fadd_rn(ic.z, __fmul_rn(s2.z, __fsub_rn(g.z, x.z)));
        vn.w = __fadd_rn(ic.w, __fmul_rn(s2.w, __fsub_rn(g.w, x.w)));
        xn.x = __fadd_rn(x.x, vn.x);
        xn.y = __fadd_rn(x.y, vn.y);
        xn.z = __fadd_rn(x.z, vn.z);
        xn.w = __fadd_rn(x.w, vn.w);
        const int64_t o = nb + 4 * (int64_t)e;
        *reinterpret_cast<float4*>(sw.pos_next + o) = xn;
        *reinterpret_cast<float4*>(sw.vel + o) = vn;
      }
    }
  } else {
    for (int e = threadIdx.x; e < Pn * d; e += kThreads) {
      const int pq = e / d, j = e - pq * d;
      const int64_t o = nb + e;
      const float x = __ldcg(sw.pos + o);
      const float vn =
          __fadd_rn(__ldcg(sw.ic + o), __fmul_rn(__ldcg(sw.s2 + o), __fsub_rn(__ldcg(gsrc + j), x)));
      sw.pos_next[o] = __fadd_rn(x, vn);
      sw.vel[o] = vn;
    }
  }
}

// Histogram and threshold scan of regression searches in the FP32 form
// (Sec. II-A, Eqs. 3-4 with the squared error): per bin the weight and the
// fixed-point sums of w (y - c) and w (y - c)^2. Shared-memory atomics are
// 32-bit only (64-bit ones run several times slower on this GPU): each
// 64-bit moment v is added as three pieces, v mod 2^16, (v >> 16) mod 2^16
// (each sum stays below 2^32 for up to 65535 entries per counter) and the
// signed v >> 32, and the bin's sum is rebuilt exactly as
// hi 2^32 + mid 2^16 + lo. Lane l adds into its particle's copy l mod
// kMseCopies (entries of one warp that fall in the same bin rarely meet at
// one address; rows
// padded by one word so equal bins of different copies sit in different
// banks). Entries are read straight from L2 with several 16-byte groups in
// flight per thread; the copies are summed, the cluster's ranks merged
// through distributed shared memory, and the scan is block_scan_mse:
// integer sums are order-free, so the scores are those of the staged-copy
// kernel. In batches of many nodes each CTA scores two particles: the
// entries' moments are read once for both (they are the same for every
// particle, only the bins differ), and the fewer CTAs carry less fixed cost
// each. The tail (score, pbest step, the next move's gB-independent
// terms) is k_hist_cls's, with its inputs prefetched.
constexpr int kMseWords = 7;  // weight; lo, mid, hi of each of the two moments
// Particles per CTA: 1 (8 copies per particle, lane mod 8), or 2 (4 copies,
// lane mod 4) for batches of many nodes, where fewer, fuller CTAs pay.
__host__ __device__ constexpr int mse_copies(int NP) { return NP == 1 ? 8 : 4; }
// CTAs (node x particle) from which a batch takes two particles per CTA.
constexpr int64_t kMsePairFrom = 4096;
__host__ __device__ inline int mse_np(const Problem& pr, int A) {
  return (int64_t)A * pr.P >= kMsePairFrom ? 2 : 1;
}
// Largest node: a counter takes the entries of one lane in mse_copies(NP)
// (plus at most about 1,100 of rounding), at most 65535 (the smaller bound).
constexpr int kMseMaxSlice = 4 * (65535 - 1100);

// 32-bit words of one particle's counters [kMseWords][copies][B + 1].
__host__ __device__ inline int mse_particle_words(int B, int NP) {
  return kMseWords * mse_copies(NP) * (B + 1);
}
// 32-bit words of the CTA's counters, also the top-k selection's scratch
// (P scores and 2 P ints), a multiple of 4.
__host__ __device__ inline int mse_count_words(int B, int P, int NP) {
  const int cells = NP * mse_particle_words(B, NP);
  const int topk = (int)((sizeof(EvalRes) + 8) * P / 4);
  return ((cells > topk ? cells : topk) + 3) & ~3;
}

template <int NP>
__global__ void __launch_bounds__(kThreads, 2)
    k_hist_mse(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes,
               const int32_t* __restrict__ list, int t, int do_update,
               const double* /* c ln c table: unused by the squared error */) {
  namespace cg = cooperative_groups;
  constexpr int kMseCopies = mse_copies(NP);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ HcScratch sc;
  __shared__ ScanScratch ss;
  __shared__ EvalRes s_pb[NP];
  __shared__ int s_imp[NP];
  const cg::cluster_group cl = cg::this_cluster();
  pdl_trigger();
  const int S = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int a = list ? list[blockIdx.x / S] : (int)blockIdx.x / S;
  const int p0 = blockIdx.y * NP;
  const int np = min(NP, pr.P - p0);  // the CTA's particles p0 .. p0 + np - 1
  const int lane = threadIdx.x & 31;
  const int B = pr.B, d = pr.d, BS = B + 1;  // copy stride (padded)
  const NodeDesc nd = nodes[a];
  const int dv = hc_dvec(d);
  // counters of particle q: [kMseWords][copies][BS] at hcnt + q * pwords
  uint32_t* hcnt = reinterpret_cast<uint32_t*>(smem);
  const int plane = kMseCopies * BS, pwords = mse_particle_words(B, NP);
  // per particle: c1 r1, c2 r2 of its next move, its x, v and pB rows
  float* rows0 = reinterpret_cast<float*>(hcnt + mse_count_words(B, pr.P, NP));
  auto row = [&](int q, int k) { return rows0 + (size_t)(5 * q + k) * dv; };
  const bool upd = do_update && rank == 0;
  const bool premove = upd && sw.ic && t < sw.T;

  for (int i = threadIdx.x; i < NP * pwords; i += kThreads) hcnt[i] = 0u;
  if (premove) {
    const uint32_t k0 = (uint32_t)sw.co.seed, k1 = (uint32_t)(sw.co.seed >> 32);
    for (int i = threadIdx.x; i < np * ((d + 3) >> 2); i += kThreads) {
      const int q = i / ((d + 3) >> 2), qq = i - q * ((d + 3) >> 2);
      const U4 r1 = philox4x32_10(nd.uid, (uint32_t)(t + 1), (uint32_t)(p0 + q),
                                  (uint32_t)qq | (kR1 << 24), k0, k1);
      const U4 r2 = philox4x32_10(nd.uid, (uint32_t)(t + 1), (uint32_t)(p0 + q),
                                  (uint32_t)qq | (kR2 << 24), k0, k1);
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (4 * qq + c < d) {
          row(q, 0)[4 * qq + c] = __fmul_rn(sw.co.c1, uniform24(r1.v[c]));
          row(q, 1)[4 * qq + c] = __fmul_rn(sw.co.c2, uniform24(r2.v[c]));
        }
    }
  }
  __syncthreads();  // the zeroed copies, before any binning
  pdl_wait();
  const int64_t ci0 = (int64_t)a * pr.Pp + p0;
  int* zz0 = sw.zmm + ci0 * 2;
  const int chunk = ((nd.seg_len + S - 1) / S + 3) & ~3;
  const int r_begin = min(nd.seg_len, rank * chunk);
  const int r_end = min(nd.seg_len, r_begin + chunk);
  const int64_t e0 = nd.seg_start + r_begin;
  const float* zs0 = sw.z + (int64_t)p0 * pr.Ez + e0;
  const float* zs1 = np > 1 ? zs0 + pr.Ez : zs0;
  const long long* m1 = pr.m1 + e0;
  const long long* m2 = pr.m2 + e0;
  const uint32_t* ws = pr.w ? pr.w + e0 : nullptr;
  const int n = r_end - r_begin;
  const bool g16 = (e0 & 3) == 0;
  const int n4 = g16 ? n >> 2 : 0;
  constexpr int U = 2;  // groups of four entries in flight per thread
  float4 zv[U][NP];
  longlong2 a1[U][2], a2[U][2];
  uint4 wv[U];
  auto load_groups = [&](int g0) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int g = g0 + u * kThreads;
      if (g < n4) {
        zv[u][0] = __ldcg(reinterpret_cast<const float4*>(zs0) + g);
        if (NP > 1) zv[u][NP - 1] = __ldcg(reinterpret_cast<const float4*>(zs1) + g);
        a1[u][0] = __ldg(reinterpret_cast<const longlong2*>(m1) + 2 * g);
        a1[u][1] = __ldg(reinterpret_cast<const longlong2*>(m1) + 2 * g + 1);
        a2[u][0] = __ldg(reinterpret_cast<const longlong2*>(m2) + 2 * g);
        a2[u][1] = __ldg(reinterpret_cast<const longlong2*>(m2) + 2 * g + 1);
        wv[u] = ws ? __ldg(reinterpret_cast<const uint4*>(ws) + g) : make_uint4(1, 1, 1, 1);
      }
    }
  };
  load_groups(threadIdx.x);
  // the tail's inputs, in flight from here: the particles' pbest scores and
  // the node's gbest score (evaluation t - 1), their x, v and pB rows
  if (upd) {
    constexpr int kResWords = (int)(sizeof(EvalRes) / 4);
    const int64_t gi = (int64_t)((t + 1) & 1) * sw.n_nodes + a;
    if (threadIdx.x < np * kResWords) {
      const int q = threadIdx.x / kResWords, w = threadIdx.x - q * kResWords;
      cp_async4(reinterpret_cast<uint32_t*>(s_pb + q) + w,
                reinterpret_cast<const uint32_t*>(sw.pb + ci0 + q) + w, 4);
    } else if (threadIdx.x >= 128 && threadIdx.x < 128 + kResWords && sw.imp) {
      cp_async4(reinterpret_cast<uint32_t*>(&sc.gb) + (threadIdx.x - 128),
                reinterpret_cast<const uint32_t*>(sw.gb + gi) + (threadIdx.x - 128), 4);
    }
    for (int i = threadIdx.x; i < np * d; i += kThreads) {
      const int q = i / d, j = i - q * d;
      const int64_t o = (ci0 + q) * d + j;
      cp_async4(row(q, 2) + j, sw.pos + o, 4);
      if (premove) {
        cp_async4(row(q, 3) + j, sw.vel + o, 4);
        cp_async4(row(q, 4) + j, sw.pbest + o, 4);
      }
    }
    cp_async_commit();
  }
  // the particles' ranges and bin widths, read by every thread (thread 0
  // resets the ranges only after the barriers below)
  float zmin[NP], inv_w[NP];
  bool ok[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    zmin[q] = 0.f;
    inv_w[q] = 0.f;
    ok[q] = false;
    if (q < np) {
      const int lo_o = __ldcg(zz0 + 2 * q), hi_o = __ldcg(zz0 + 2 * q + 1);
      if (lo_o != INT_MAX) {
        const float lo = ord2f(lo_o), hi = ord2f(hi_o);
        inv_w[q] = __fdiv_rn((float)B, __fsub_rn(hi, lo));
        zmin[q] = lo;
        ok[q] = (hi > lo) && isfinite(inv_w[q]);
      }
    }
  }
  // ---- binning of this rank's slice, both particles from one read of the
  // entries' moments
  {
    const int cpy = (lane % kMseCopies) * BS;
    auto add = [&](int q, float z, long long v1, long long v2, uint32_t w) {
      uint32_t* h = hcnt + q * pwords + cpy + bin_of(z, zmin[q], inv_w[q], B);
      const unsigned long long u1 = (unsigned long long)v1, u2 = (unsigned long long)v2;
      atomicAdd(h, w);
      atomicAdd(h + plane, (uint32_t)(u1 & 0xffffu));
      atomicAdd(h + 2 * plane, (uint32_t)((u1 >> 16) & 0xffffu));
      atomicAdd(h + 3 * plane, (uint32_t)(u1 >> 32));  // the signed high word, mod 2^32
      atomicAdd(h + 4 * plane, (uint32_t)(u2 & 0xffffu));
      atomicAdd(h + 5 * plane, (uint32_t)((u2 >> 16) & 0xffffu));
      atomicAdd(h + 6 * plane, (uint32_t)(u2 >> 32));
    };
    if (ok[0] || ok[NP - 1]) {
      for (int g0 = threadIdx.x; g0 < n4; g0 += U * kThreads) {
        if (g0 != (int)threadIdx.x) load_groups(g0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (g0 + u * kThreads >= n4) break;
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            if (!ok[q]) continue;
            add(q, zv[u][q].x, a1[u][0].x, a2[u][0].x, wv[u].x);
            add(q, zv[u][q].y, a1[u][0].y, a2[u][0].y, wv[u].y);
            add(q, zv[u][q].z, a1[u][1].x, a2[u][1].x, wv[u].z);
            add(q, zv[u][q].w, a1[u][1].y, a2[u][1].y, wv[u].w);
          }
        }
      }
      for (int i = (n4 << 2) + (int)threadIdx.x; i < n; i += kThreads) {
        const long long v1 = __ldg(m1 + i), v2 = __ldg(m2 + i);
        const uint32_t w = ws ? __ldg(ws + i) : 1u;
        if (ok[0]) add(0, __ldcg(zs0 + i), v1, v2, w);
        if (NP > 1 && ok[NP - 1]) add(NP - 1, __ldcg(zs1 + i), v1, v2, w);
      }
    }
  }
  __syncthreads();
  // ---- each particle's copies into bin sums (thread b: bin b), written
  // after every thread has read the copies: the weight into the particle's
  // first row, the moments rebuilt exactly as 64-bit integers (two's
  // complement: signed sums wrap exactly) over its first piece plane
  uint32_t w[NP];
  unsigned long long v[NP][2];
  const int bi = threadIdx.x;  // B <= kThreads
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    w[q] = 0;
    v[q][0] = v[q][1] = 0ull;
    if (bi < B && q < np) {
#pragma unroll
      for (int c = 0; c < kMseCopies; ++c) {
        const uint32_t* h = hcnt + q * pwords + c * BS + bi;
        w[q] += h[0];
#pragma unroll
        for (int m = 0; m < 2; ++m)
          v[q][m] += (unsigned long long)h[(1 + 3 * m) * plane] +
                     ((unsigned long long)h[(2 + 3 * m) * plane] << 16) +
                     ((unsigned long long)(long long)(int32_t)h[(3 + 3 * m) * plane] << 32);
      }
    }
  }
  __syncthreads();
  auto hw_of = [&](int q) { return hcnt + q * pwords; };  // [B]
  auto hs_of = [&](int q) {                                  // [2][B]
    return reinterpret_cast<unsigned long long*>(hcnt + q * pwords + ((plane + 1) & ~1));
  };
#pragma unroll
  for (int q = 0; q < NP; ++q)
    if (bi < B && q < np) {
      hw_of(q)[bi] = w[q];
      hs_of(q)[bi] = v[q][0];
      hs_of(q)[B + bi] = v[q][1];
    }
  // ---- the cluster's bins into rank 0: rank r sums the r-th of S slices
  // of the bins over every rank and stores the sums into rank 0's
  if (S > 1) {
    cl.sync();  // every rank's bin sums are complete
    const int per = (B + S - 1) / S;
    const int lo = rank * per, hi = min(B, lo + per);
    for (int q = 0; q < np; ++q)
      for (int i = lo + (int)threadIdx.x; i < hi; i += kThreads) {
        uint32_t ww = 0;
        unsigned long long v1 = 0ull, v2 = 0ull;
#pragma unroll
        for (int r = 0; r < 16; ++r)
          if (r < S) {
            ww += cl.map_shared_rank(hw_of(q), r)[i];
            v1 += cl.map_shared_rank(hs_of(q), r)[i];
            v2 += cl.map_shared_rank(hs_of(q), r)[B + i];
          }
        cl.map_shared_rank(hw_of(q), 0)[i] = ww;
        cl.map_shared_rank(hs_of(q), 0)[i] = v1;
        cl.map_shared_rank(hs_of(q), 0)[B + i] = v2;
      }
    cl.sync();  // rank 0's bins are complete; no rank reads another's
    if (rank != 0) return;
  }
  cp_async_wait<0>();  // the tail's prefetched inputs
  __syncthreads();
  EvalRes res[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    res[q] = invalid_res();
    if (q < np && ok[q]) {  // the same branch in every thread (block_scan_mse syncs)
      res[q] = block_scan_mse(hw_of(q), reinterpret_cast<const long long*>(hs_of(q)),
                              reinterpret_cast<const long long*>(hs_of(q) + B),
                              pr.mscale[2 * a], pr.mscale[2 * a + 1], B, pr.min_leaf, ss);
      res[q].zmin = zmin[q];
      res[q].inv_w = inv_w[q];
    }
  }
  // ---- scores, range resets, pbest steps, the next moves' gB-independent terms
  if (threadIdx.x == 0) {
    for (int q = 0; q < np; ++q) {
      const int64_t ci = ci0 + q;
      sw.cur[ci] = res[q];
      zz0[2 * q] = INT_MAX;  // ready for the next iteration
      zz0[2 * q + 1] = INT_MIN;
      int imp = 0;
      if (do_update) {
        if (sw.imp && res[q].valid && (t == 0 || better(res[q], sc.gb, pr.crit)))
          atomicOr(sw.imp + (int64_t)(t & 1) * sw.n_nodes + a, 1);
        imp = (t == 0) || better(res[q], s_pb[q], pr.crit);
        if (imp) sw.pb[ci] = res[q];
      }
      s_imp[q] = imp;
    }
  }
  if (sw.tk_sel) {
    // the reduced pass of the BF16 form: the last CTA of the node to score
    // its particles selects the node's top k (the counters are free by now)
    __threadfence();  // this CTA's score writes before the count
    __syncthreads();
    if (threadIdx.x == 0) sc.ok = atomicAdd(&sw.done[a], np) + np == pr.P;
    __syncthreads();
    if (sc.ok) {
      __threadfence();
      topk_select(pr, sw, a, reinterpret_cast<unsigned char*>(hcnt));
      if (threadIdx.x == 0) sw.done[a] = 0;
    }
  }
  if (!do_update) return;
  __syncthreads();
  for (int i = threadIdx.x; i < np * d; i += kThreads) {
    const int q = i / d, j = i - q * d;
    const bool imp = s_imp[q];
    if (!imp && !premove) continue;
    const int64_t o = (ci0 + q) * d + j;
    const float x = row(q, 2)[j];
    if (imp) sw.pbest[o] = x;  // the position is kept on improvement
    if (premove) {
      // ic = omega v + (c1 r1)(pB - x); pB is x itself after an improvement
      const float pbv = imp ? x : row(q, 4)[j];
      sw.ic[o] = __fadd_rn(__fmul_rn(sw.co.inertia, row(q, 3)[j]),
                           __fmul_rn(row(q, 0)[j], __fsub_rn(pbv, x)));
      sw.s2[o] = row(q, 1)[j];
    }
  }
}

const void* hist_cls_fn(const Problem& pr, int np = 1) {
  return pr.crit == SLM_GINI      ? (const void*)k_hist_cls<SLM_GINI>
         : pr.crit == SLM_ENTROPY ? (const void*)k_hist_cls<SLM_ENTROPY>
         : np == 2                ? (const void*)k_hist_mse<2>
                                  : (const void*)k_hist_mse<1>;
}

size_t hist_cls_smem(const Problem& pr, int np = 1) {
  const size_t tail = sizeof(float) * 5 * (size_t)hc_dvec(pr.d);
  if (pr.crit == SLM_MSE) return (size_t)mse_count_words(pr.B, pr.P, np) * 4 + np * tail;
  return sizeof(uint32_t) * (size_t)hc_words(pr.B, pr.K, pr.P) + tail;
}

}  // namespace

bool hist_cls_ok(const Problem& pr) {
  if (pr.B < 2 || pr.B > kThreads || hist_cls_smem(pr, 1) > 200 * 1024 ||
      hist_cls_smem(pr, 2) > 200 * 1024)
    return false;
  if (pr.crit == SLM_MSE) return pr.m1 && pr.m2 && pr.mscale;
  return pr.lab && pr.K >= 1 && pr.K <= kMaxClasses;
}

bool hist_cls_fits(const Problem& pr, int64_t max_len) {
  return pr.crit != SLM_MSE || max_len <= kMseMaxSlice;
}

cudaError_t prepare_hist_cls(const Problem& pr) {
  for (int np = 1; np <= (pr.crit == SLM_MSE ? 2 : 1); ++np) {
    const void* f = hist_cls_fn(pr, np);
    cudaError_t e = allow_smem((const void*)f, (int)hist_cls_smem(pr, np));
    if (!e) e = allow_cluster((const void*)f);
    if (e) return e;
  }
  return cudaSuccess;
}

int hist_cls_split(const Problem& pr, int A, int64_t max_len, int n_sm) {
  const int np = pr.crit == SLM_MSE ? mse_np(pr, A) : 1;
  int per_sm = 1;
  if (occupancy(&per_sm, hist_cls_fn(pr, np), kThreads, hist_cls_smem(pr, np)) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  // up to one wave of resident CTAs, slices of at least 1024 entries, at
  // most 8 CTAs per cluster (the portable size)
  const int64_t resident = (int64_t)(per_sm > 0 ? per_sm : 1) * n_sm;
  int S = 1;
  const int64_t ctas = (pr.P + np - 1) / np;  // per node and slice
  while (2 * S <= 8 && (int64_t)A * ctas * (2 * S) <= resident && max_len / (2 * S) >= 1024) S *= 2;
  return S;
}

cudaError_t launch_hist_cls(const Problem& pr, const Swarm& sw, const NodeDesc* nodes, int A,
                            int S, int t, int do_update, const double* xtab, cudaStream_t st,
                            const int32_t* list) {
  if (A <= 0) return cudaSuccess;
  const int np = pr.crit == SLM_MSE ? mse_np(pr, A) : 1;  // particles per CTA
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(A * S), (unsigned)((pr.P + np - 1) / np), 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = hist_cls_smem(pr, np);
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  const void* f = hist_cls_fn(pr, np);
  void* args[] = {(void*)&pr, (void*)&sw, (void*)&nodes, (void*)&list, (void*)&t,
                  (void*)&do_update, (void*)&xtab};
  return cudaLaunchKernelExC(&cfg, f, args);
}

}  // namespace slm
