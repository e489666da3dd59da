// Block-wide threshold scans shared by the histogram kernels (Sec. II-A,
// Eqs. 3-4): the scratch they use, the edge order (ties to the lower edge)
// and the regression scan over fixed-point bin moments; and the reduced
// pass's top-k selection of the BF16 form, which the last histogram CTA of
// a node runs.
#pragma once

#include <cuda_runtime.h>

#include "device_util.cuh"
#include "slm_internal.cuh"

namespace slm {
namespace {

// Shared scratch of the block-wide scans.
struct ScanScratch {
  uint32_t nl[kMaxBins];  // left weight of each edge (classification)
  uint32_t pc[kMaxBins];  // MSE prefix: weight
  long long ps[kMaxBins];  // MSE prefix: fixed-point sum w (y-c)
  long long pq[kMaxBins];  // MSE prefix: fixed-point sum w (y-c)^2
  uint64_t wn[kThreads / 32], wd[kThreads / 32];
  double wl[kThreads / 32];
  int wb[kThreads / 32];
  EvalRes res;
};

// Ties: the lower edge. Gini scores are rationals n/d (larger is better),
// the others losses (smaller is better).
template <int CRIT>
__device__ __forceinline__ bool edge_takes(uint64_t on, uint64_t od, double ol, int ob, uint64_t bn,
                                           uint64_t bd, double bl, int bb) {
  if (ob < 0) return false;
  if (bb < 0) return true;
  if (CRIT == SLM_GINI) return prod_gt(on, bd, bn, od) || (!prod_gt(bn, od, on, bd) && ob < bb);
  return ol < bl || (!(bl < ol) && ob < bb);
}

// Block-wide argmin over the threads' candidates (bb < 0: none); the winner
// lands in sc.wn[0] / sc.wd[0] / sc.wl[0] / sc.wb[0].
template <int CRIT>
__device__ __forceinline__ void block_argmin(uint64_t bn, uint64_t bd, double bl, int bb,
                                             ScanScratch& sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const int ob = __shfl_xor_sync(0xffffffffu, bb, off);
    const uint64_t on = __shfl_xor_sync(0xffffffffu, bn, off);
    const uint64_t od = __shfl_xor_sync(0xffffffffu, bd, off);
    const double ol = __shfl_xor_sync(0xffffffffu, bl, off);
    if (edge_takes<CRIT>(on, od, ol, ob, bn, bd, bl, bb)) {
      bn = on;
      bd = od;
      bl = ol;
      bb = ob;
    }
  }
  if (lane == 0) {
    sc.wn[warp] = bn;
    sc.wd[warp] = bd;
    sc.wl[warp] = bl;
    sc.wb[warp] = bb;
  }
  __syncthreads();
  if (warp == 0) {
    const bool in = lane < kThreads / 32;
    bn = in ? sc.wn[lane] : 0;
    bd = in ? sc.wd[lane] : 0;
    bl = in ? sc.wl[lane] : 0.0;
    bb = in ? sc.wb[lane] : -1;
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) {
      const int ob = __shfl_xor_sync(0xffffffffu, bb, off);
      const uint64_t on = __shfl_xor_sync(0xffffffffu, bn, off);
      const uint64_t od = __shfl_xor_sync(0xffffffffu, bd, off);
      const double ol = __shfl_xor_sync(0xffffffffu, bl, off);
      if (edge_takes<CRIT>(on, od, ol, ob, bn, bd, bl, bb)) {
        bn = on;
        bd = od;
        bl = ol;
        bb = ob;
      }
    }
    if (lane == 0) {
      sc.wn[0] = bn;
      sc.wd[0] = bd;
      sc.wl[0] = bl;
      sc.wb[0] = bb;
    }
  }
  __syncthreads();
}

// Regression threshold scan of one particle by the whole CTA. cnt/s/q: [B]
// weight, sum w y, sum w y^2. Prefix sums by warp 0 (sequential within a
// lane, then across lanes), then one thread per edge.
// s[b], q[b]: fixed-point sums of w (y-c) and w (y-c)^2 of bin b, worth
// f1 and f2 per unit; prefix sums stay exact integers and become doubles
// per edge: SSE of a side = Q - S^2 / n (centred, so little cancels).
__device__ EvalRes block_scan_mse(const uint32_t* cnt, const long long* s, const long long* q,
                                  double f1, double f2, int B, int min_leaf, ScanScratch& sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    const int bpl = (B + 31) >> 5;
    uint32_t cs = 0;
    long long ss = 0, qs = 0;
    for (int i = 0; i < bpl; ++i) {
      const int j = lane * bpl + i;
      if (j < B) {
        cs += cnt[j];
        ss += s[j];
        qs += q[j];
      }
    }
    uint32_t ic = cs;
    long long is = ss, iq = qs;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t vc = __shfl_up_sync(0xffffffffu, ic, off);
      const long long vs = __shfl_up_sync(0xffffffffu, is, off);
      const long long vq = __shfl_up_sync(0xffffffffu, iq, off);
      if (lane >= off) {
        ic += vc;
        is = vs + is;
        iq = vq + iq;
      }
    }
    // exclusive prefix = the previous lane's inclusive sums
    uint32_t rc = ic - cs;
    long long rs = __shfl_up_sync(0xffffffffu, is, 1);
    long long rq = __shfl_up_sync(0xffffffffu, iq, 1);
    if (lane == 0) {
      rs = 0;
      rq = 0;
    }
    for (int i = 0; i < bpl; ++i) {
      const int j = lane * bpl + i;
      if (j < B) {
        rc += cnt[j];
        rs += s[j];
        rq += q[j];
        sc.pc[j] = rc;
        sc.ps[j] = rs;
        sc.pq[j] = rq;
      }
    }
  }
  __syncthreads();
  const uint32_t ntot = sc.pc[B - 1];
  const long long stot = sc.ps[B - 1], qtot = sc.pq[B - 1];
  const int b = 1 + threadIdx.x;
  double bl = 0.0;
  int bb = -1;
  if (b < B && cnt[b - 1] != 0) {  // empty bin b-1: same partition as edge b-1
    const uint32_t nl = sc.pc[b - 1], nr = ntot - nl;
    if (nl >= (uint32_t)min_leaf && nr >= (uint32_t)min_leaf) {
      const double sl = (double)sc.ps[b - 1] * f1, ql = (double)sc.pq[b - 1] * f2;
      const double sr = (double)(stot - sc.ps[b - 1]) * f1;
      const double qr = (double)(qtot - sc.pq[b - 1]) * f2;
      const double sse_l = ql - sl * sl / (double)nl;
      const double sse_r = qr - sr * sr / (double)nr;
      bl = (sse_l + sse_r) / (double)ntot;
      bb = b;
    }
  }
  block_argmin<SLM_MSE>(0, 0, bl, bb, sc);
  if (threadIdx.x == 0) {
    EvalRes res = invalid_res();
    const int wb = sc.wb[0];
    if (wb >= 0) {
      res.valid = 1;
      res.bin = wb;
      res.nl = sc.pc[wb - 1];
      res.nr = ntot - sc.pc[wb - 1];
      res.loss = sc.wl[0];
    }
    sc.res = res;
  }
  __syncthreads();
  return sc.res;
}

// ---- top-k selection (SLM_PROJ_BF16_TOPK) ------------------------------------------

// The whole CTA selects node a's tk_k best particles by sw.cur (ties to the
// lower index; rank = particles strictly better, or equal and lower) and
// gathers their positions. scratch: P EvalRes + 2 P ints of shared memory.
__device__ __noinline__ void topk_select(const Problem& pr, const Swarm& sw, int a,
                                         unsigned char* scratch) {
  EvalRes* s_sc = reinterpret_cast<EvalRes*>(scratch);
  int* s_take = reinterpret_cast<int*>(s_sc + pr.P);
  int* s_sel = s_take + pr.P;
  const int P = pr.P, Pp = pr.Pp, d = pr.d, k = sw.tk_k, kp = sw.tk_kp;
  for (int p = threadIdx.x; p < P; p += blockDim.x) s_sc[p] = ldcg_res(sw.cur + (int64_t)a * Pp + p);
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const EvalRes me = s_sc[p];
    int rank = 0;
    for (int q = 0; q < P; ++q) {
      if (q == p) continue;
      const EvalRes o = s_sc[q];
      if (better(o, me, pr.crit) || (q < p && !better(me, o, pr.crit))) ++rank;
    }
    s_take[p] = rank < k;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < Pp; p += blockDim.x) {
    int q = -1;
    if (p < P && s_take[p]) {
      q = 0;
      for (int j = 0; j < p; ++j) q += s_take[j];
      s_sel[q] = p;
      sw.tk_sel[(int64_t)a * k + q] = p;
    }
    sw.tk_inv[(int64_t)a * Pp + p] = q;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kp * d; e += blockDim.x) {
    const int q = e / d, j = e - q * d;
    sw.tk_pos[((int64_t)a * kp + q) * d + j] =
        q < k ? sw.pos[((int64_t)a * Pp + s_sel[q]) * d + j] : 0.0f;
  }
}

}  // namespace
}  // namespace slm
