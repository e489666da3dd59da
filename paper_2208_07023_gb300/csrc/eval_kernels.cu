// Swarm scoring and update kernels.
//
// Scoring one particle on one node (Sec. II-A, Eqs. 1, 3-4; Sec. IV):
//   z_s   = a^T x_s                       one fmaf per feature, j = 0..d-1
//   bin_s = min(B-1, floor((z_s - zmin) * inv_w)),  inv_w = B / (zmax - zmin)
//   histogram of (bin, class) -- or (bin; weight, sum w y, sum w y^2)
//   every interior edge b = 1..B-1 splits bins < b | bins >= b; the weighted
//   child impurity of each admissible edge is scored and the minimum kept.
// Swarm update (Sec. III-A, Eq. pso-1; Algorithm 1):
//   v <- omega v + (c1 r1)(pB - x) + (c2 r2)(gB - x);   x <- x + v
//
// Tiling. A CTA scores kPG = 16 particles of one node. Samples are staged in
// tiles of kTS = 256 rows (gathered through the node's sample index) and the
// features in chunks of kKC = 32, in shared memory with a padded row stride.
// Each thread owns a 4 x 4 register tile (samples w*32 + sg + 8i, particles
// pg + 4j) and accumulates over the features in increasing order, so every z
// is the same sequence of fused multiply-adds whatever the tiling.
// Nodes with <= kSmallMax entries are scored by one CTA per particle group
// in one launch (two passes over the node: range, then histogram and scan).
// Larger nodes are cut into kChunk-entry work items: a range kernel (global
// ordered-int atomics), a histogram kernel writing dense per-item partial
// histograms, and a per-particle reduce-and-scan kernel.
#include <cuda_runtime.h>
#include <float.h>
#include <limits.h>
#include <math.h>

#include "philox.cuh"
#include "slm_internal.cuh"

namespace slm {

namespace {

// ---- small helpers -----------------------------------------------------------

__device__ __forceinline__ int f2ord(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) {
  return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}

// a*b > c*d on unsigned 128-bit products.
__device__ __forceinline__ bool prod_gt(uint64_t a, uint64_t b, uint64_t c,
                                        uint64_t d) {
  const uint64_t h1 = __umul64hi(a, b), l1 = a * b;
  const uint64_t h2 = __umul64hi(c, d), l2 = c * d;
  return h1 > h2 || (h1 == h2 && l1 > l2);
}

// Strictly lower loss? Gini compares the exact rationals Q = num/den (larger
// Q = lower loss); entropy and MSE compare the double loss.
__device__ __forceinline__ bool better(const EvalRes& a, const EvalRes& b,
                                       int crit) {
  if (!a.valid) return false;
  if (!b.valid) return true;
  if (crit == SLM_GINI) return prod_gt(a.num, b.den, b.num, a.den);
  return a.loss < b.loss;
}

__device__ __forceinline__ EvalRes invalid_res() {
  EvalRes r;
  r.loss = __longlong_as_double(0x7ff0000000000000LL);  // +inf
  r.num = 0;
  r.den = 0;
  r.zmin = 0.f;
  r.inv_w = 0.f;
  r.bin = -1;
  r.valid = 0;
  r.nl = 0;
  r.nr = 0;
  return r;
}

__device__ __forceinline__ EvalRes shfl_res(const EvalRes& a, int src) {
  EvalRes r;
  r.loss = __shfl_sync(0xffffffffu, a.loss, src);
  r.num = __shfl_sync(0xffffffffu, a.num, src);
  r.den = __shfl_sync(0xffffffffu, a.den, src);
  r.zmin = __shfl_sync(0xffffffffu, a.zmin, src);
  r.inv_w = __shfl_sync(0xffffffffu, a.inv_w, src);
  r.bin = __shfl_sync(0xffffffffu, a.bin, src);
  r.valid = __shfl_sync(0xffffffffu, a.valid, src);
  r.nl = __shfl_sync(0xffffffffu, a.nl, src);
  r.nr = __shfl_sync(0xffffffffu, a.nr, src);
  return r;
}

// Lexicographic (score, bin): the lowest edge among equal scores.
__device__ __forceinline__ bool edge_first(const EvalRes& a, const EvalRes& b,
                                           int crit) {
  if (better(a, b, crit)) return true;
  if (better(b, a, crit)) return false;
  return a.valid && b.valid && a.bin < b.bin;
}

__device__ __forceinline__ double xlogx(uint32_t c) {
  const double x = (double)c;
  return c ? x * log(x) : 0.0;
}

__device__ __forceinline__ int bin_of(float z, float zmin, float inv_w, int B) {
  const float off = __fsub_rn(z, zmin);
  const float pos = __fmul_rn(off, inv_w);
  int b = (int)floorf(pos);
  b = b > B - 1 ? B - 1 : b;
  return b < 0 ? 0 : b;
}

// ---- shared-memory layout of the scoring kernels ------------------------------

struct Smem {
  float* xs;       // [kTS][kXS]
  float* as;       // [kPG][kXS]
  int32_t* tidx;   // [kTS]  global sample index of each tile row
  int32_t* tlab;   // [kTS]  label (classification)
  float* ty;       // [kTS]  target (MSE)
  uint32_t* tw;    // [kTS]  multiplicity
  int* smin;       // [kPG]  ordered-int range
  int* smax;       // [kPG]
  float* zmin;     // [kPG]
  float* inv_w;    // [kPG]
  int* ok;         // [kPG]
  uint32_t* hist;  // classification [kPG][B*K]; MSE counts [kPG][B]
  double* hs;      // MSE [kPG][B]
  double* hq;      // MSE [kPG][B]
};

__host__ __device__ inline size_t hist_bytes(int crit, int B, int K) {
  return crit == SLM_MSE ? (size_t)kPG * B * (4 + 8 + 8)
                         : (size_t)kPG * B * K * 4;
}

__host__ __device__ inline size_t fixed_bytes() {
  return sizeof(float) * (kTS * kXS + kPG * kXS) + sizeof(int32_t) * kTS * 4 +
         sizeof(int) * kPG * 5;
}

__device__ __forceinline__ Smem carve(unsigned char* base, int crit, int B,
                                      int K) {
  Smem s;
  unsigned char* p = base;
  if (crit == SLM_MSE) {  // doubles first for alignment
    s.hs = (double*)p;
    p += sizeof(double) * kPG * B;
    s.hq = (double*)p;
    p += sizeof(double) * kPG * B;
    s.hist = (uint32_t*)p;
    p += sizeof(uint32_t) * kPG * B;
  } else {
    s.hs = s.hq = nullptr;
    s.hist = (uint32_t*)p;
    p += sizeof(uint32_t) * kPG * B * K;
  }
  p = (unsigned char*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
  s.xs = (float*)p;
  p += sizeof(float) * kTS * kXS;
  s.as = (float*)p;
  p += sizeof(float) * kPG * kXS;
  s.tidx = (int32_t*)p;
  p += sizeof(int32_t) * kTS;
  s.tlab = (int32_t*)p;
  s.ty = (float*)p;
  p += sizeof(int32_t) * kTS;
  s.tw = (uint32_t*)p;
  p += sizeof(uint32_t) * kTS;
  s.smin = (int*)p;
  p += sizeof(int) * kPG;
  s.smax = (int*)p;
  p += sizeof(int) * kPG;
  s.zmin = (float*)p;
  p += sizeof(float) * kPG;
  s.inv_w = (float*)p;
  p += sizeof(float) * kPG;
  s.ok = (int*)p;
  return s;
}

// Loads tile rows [r0, r0 + n) of a node segment: sample index, label or
// target, and multiplicity.
__device__ __forceinline__ void load_tile_meta(const Problem& pr, const Smem& s,
                                               int64_t e0, int n) {
  for (int r = threadIdx.x; r < kTS; r += kThreads) {
    if (r < n) {
      const int64_t e = e0 + r;
      const int32_t si = pr.idx[e];
      s.tidx[r] = si;
      if (pr.crit == SLM_MSE)
        s.ty[r] = pr.y[si];
      else
        s.tlab[r] = pr.labels[si];
      s.tw[r] = pr.w ? pr.w[e] : 1u;
    } else {
      s.tidx[r] = -1;
      s.tw[r] = 0;
      if (pr.crit == SLM_MSE)
        s.ty[r] = 0.f;
      else
        s.tlab[r] = 0;
    }
  }
}

// z for the tile's rows x the group's 16 particles. Requires tile meta loaded
// and a __syncthreads() since. pos: [kPG, d] positions of the group.
__device__ __forceinline__ void project_tile(const Problem& pr, const Smem& s,
                                             const float* __restrict__ pos,
                                             int n, float acc[4][4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sg = lane & 7, pg = lane >> 3;
  const int d = pr.d;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;

  for (int k0 = 0; k0 < d; k0 += kKC) {
    const int kc = min(kKC, d - k0);
    const int kc4 = (kc + 3) & ~3;
    __syncthreads();  // previous chunk fully consumed
    for (int e = threadIdx.x; e < kTS * kc4; e += kThreads) {
      const int r = e / kc4, c = e - r * kc4;
      float v = 0.0f;
      if (r < n && c < kc) v = __ldg(pr.X + (int64_t)s.tidx[r] * d + k0 + c);
      s.xs[r * kXS + c] = v;
    }
    for (int e = threadIdx.x; e < kPG * kc4; e += kThreads) {
      const int p = e / kc4, c = e - p * kc4;
      s.as[p * kXS + c] = c < kc ? pos[(int64_t)p * d + k0 + c] : 0.0f;
    }
    __syncthreads();
    const float* xr = s.xs + (warp * 32 + sg) * kXS;
    const float* ar = s.as + pg * kXS;
    for (int c = 0; c < kc4; c += 4) {
      float4 xv[4], av[4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        xv[i] = *reinterpret_cast<const float4*>(xr + i * 8 * kXS + c);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        av[j] = *reinterpret_cast<const float4*>(ar + j * 4 * kXS + c);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j] = fmaf(xv[i].x, av[j].x, acc[i][j]);
          acc[i][j] = fmaf(xv[i].y, av[j].y, acc[i][j]);
          acc[i][j] = fmaf(xv[i].z, av[j].z, acc[i][j]);
          acc[i][j] = fmaf(xv[i].w, av[j].w, acc[i][j]);
        }
    }
  }
}

// Range of each particle over the tile's valid rows, folded into s.smin/smax.
__device__ __forceinline__ void tile_minmax(const Smem& s, int n,
                                            const float acc[4][4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sg = lane & 7, pg = lane >> 3;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float lo = FLT_MAX, hi = -FLT_MAX;
    bool any = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = warp * 32 + sg + 8 * i;
      if (r < n) {
        const float z = acc[i][j];
        lo = z < lo ? z : lo;
        hi = z > hi ? z : hi;
        any = true;
      }
    }
    int olo = any ? f2ord(lo) : INT_MAX, ohi = any ? f2ord(hi) : INT_MIN;
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
      olo = min(olo, __shfl_xor_sync(0xffffffffu, olo, off));
      ohi = max(ohi, __shfl_xor_sync(0xffffffffu, ohi, off));
    }
    if (sg == 0 && olo != INT_MAX) {
      atomicMin(&s.smin[pg + 4 * j], olo);
      atomicMax(&s.smax[pg + 4 * j], ohi);
    }
  }
}

// Bins the tile's z and adds them to the shared histograms.
__device__ __forceinline__ void tile_hist(const Problem& pr, const Smem& s,
                                          int n, int p_base,
                                          const float acc[4][4],
                                          int32_t* bins_out, int64_t n_idx,
                                          int64_t row0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sg = lane & 7, pg = lane >> 3;
  const int B = pr.B, K = pr.K;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int pl = pg + 4 * j;
    if (p_base + pl >= pr.P || !s.ok[pl]) continue;
    const float zmin = s.zmin[pl], inv_w = s.inv_w[pl];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = warp * 32 + sg + 8 * i;
      if (r >= n) continue;
      const int b = bin_of(acc[i][j], zmin, inv_w, B);
      const uint32_t w = s.tw[r];
      if (pr.crit == SLM_MSE) {
        const double wy = (double)w * (double)s.ty[r];
        atomicAdd(&s.hist[pl * B + b], w);
        atomicAdd(&s.hs[pl * B + b], wy);
        atomicAdd(&s.hq[pl * B + b], wy * (double)s.ty[r]);
      } else {
        atomicAdd(&s.hist[(pl * B + b) * K + s.tlab[r]], w);
      }
      if (bins_out) bins_out[(int64_t)(p_base + pl) * n_idx + row0 + r] = b;
    }
  }
}

// ---- threshold scans (one warp, one particle) ----------------------------------

constexpr int kMaxBPL = kMaxBins / 32;

// Classification. h: [B][K] counts of one particle.
__device__ EvalRes scan_cls(const uint32_t* h, int B, int K, int min_leaf,
                            int crit) {
  const int lane = threadIdx.x & 31;
  const int BPL = (B + 31) >> 5;
  const int j0 = lane * BPL;
  uint32_t nL[kMaxBPL];
  uint64_t SL[kMaxBPL], SR[kMaxBPL];
  double hL[kMaxBPL], hR[kMaxBPL];
#pragma unroll
  for (int i = 0; i < kMaxBPL; ++i) {
    nL[i] = 0;
    SL[i] = SR[i] = 0;
    hL[i] = hR[i] = 0.0;
  }
  uint32_t ntot = 0;
  for (int k = 0; k < K; ++k) {
    uint32_t c[kMaxBPL];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kMaxBPL; ++i) {
      const int j = j0 + i;
      c[i] = (i < BPL && j < B) ? h[j * K + k] : 0u;
      sum += c[i];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
    ntot += tot;
    uint32_t run = incl - sum;
#pragma unroll
    for (int i = 0; i < kMaxBPL; ++i) {
      if (i >= BPL) break;
      run += c[i];
      const uint32_t rr = tot - run;
      nL[i] += run;
      if (crit == SLM_GINI) {
        SL[i] += (uint64_t)run * run;
        SR[i] += (uint64_t)rr * rr;
      } else {
        hL[i] += xlogx(run);
        hR[i] += xlogx(rr);
      }
    }
  }
  EvalRes best = invalid_res();
#pragma unroll
  for (int i = 0; i < kMaxBPL; ++i) {
    if (i >= BPL) break;
    const int b = j0 + i + 1;
    if (b > B - 1) break;
    const uint32_t nl = nL[i], nr = ntot - nl;
    if (nl < (uint32_t)min_leaf || nr < (uint32_t)min_leaf) continue;
    EvalRes c = invalid_res();
    c.valid = 1;
    c.bin = b;
    c.nl = nl;
    c.nr = nr;
    if (crit == SLM_GINI) {
      const uint64_t num = SL[i] * nr + SR[i] * nl;
      const uint64_t den = (uint64_t)nl * nr;
      const uint64_t nden = (uint64_t)ntot * den;
      c.num = num;
      c.den = den;
      c.loss = (double)(nden - num) / (double)nden;
    } else {
      const double hh = (xlogx(nl) - hL[i]) + (xlogx(nr) - hR[i]);
      c.loss = hh / (double)ntot;
    }
    if (better(c, best, crit)) best = c;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const EvalRes o = shfl_res(best, lane ^ off);
    if (edge_first(o, best, crit)) best = o;
  }
  return best;
}

// Regression. cnt/s/q: [B] weight, sum w y, sum w y^2 of one particle.
__device__ EvalRes scan_mse(const uint32_t* cnt, const double* s,
                            const double* q, int B, int min_leaf) {
  const int lane = threadIdx.x & 31;
  const int BPL = (B + 31) >> 5;
  const int j0 = lane * BPL;
  uint32_t c[kMaxBPL];
  double sv[kMaxBPL], qv[kMaxBPL];
  uint32_t cs = 0;
  double ss = 0.0, qs = 0.0;
#pragma unroll
  for (int i = 0; i < kMaxBPL; ++i) {
    const int j = j0 + i;
    const bool in = i < BPL && j < B;
    c[i] = in ? cnt[j] : 0u;
    sv[i] = in ? s[j] : 0.0;
    qv[i] = in ? q[j] : 0.0;
    cs += c[i];
    ss += sv[i];
    qs += qv[i];
  }
  uint32_t ic = cs;
  double is = ss, iq = qs;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t vc = __shfl_up_sync(0xffffffffu, ic, off);
    const double vs = __shfl_up_sync(0xffffffffu, is, off);
    const double vq = __shfl_up_sync(0xffffffffu, iq, off);
    if (lane >= off) {
      ic += vc;
      is = vs + is;
      iq = vq + iq;
    }
  }
  const uint32_t ntot = __shfl_sync(0xffffffffu, ic, 31);
  const double stot = __shfl_sync(0xffffffffu, is, 31);
  const double qtot = __shfl_sync(0xffffffffu, iq, 31);
  // exclusive prefix = the previous lane's inclusive sums
  uint32_t rc = ic - cs;
  double rs = __shfl_up_sync(0xffffffffu, is, 1);
  double rq = __shfl_up_sync(0xffffffffu, iq, 1);
  if (lane == 0) {
    rs = 0.0;
    rq = 0.0;
  }
  EvalRes best = invalid_res();
#pragma unroll
  for (int i = 0; i < kMaxBPL; ++i) {
    if (i >= BPL) break;
    rc += c[i];
    rs += sv[i];
    rq += qv[i];
    const int b = j0 + i + 1;
    if (b > B - 1) break;
    const uint32_t nl = rc, nr = ntot - rc;
    if (nl < (uint32_t)min_leaf || nr < (uint32_t)min_leaf) continue;
    const double sr = stot - rs, qr = qtot - rq;
    const double sse_l = rq - rs * rs / (double)nl;
    const double sse_r = qr - sr * sr / (double)nr;
    EvalRes e = invalid_res();
    e.valid = 1;
    e.bin = b;
    e.nl = nl;
    e.nr = nr;
    e.loss = (sse_l + sse_r) / (double)ntot;
    if (better(e, best, SLM_MSE)) best = e;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const EvalRes o = shfl_res(best, lane ^ off);
    if (edge_first(o, best, SLM_MSE)) best = o;
  }
  return best;
}

__device__ __forceinline__ void zero_hist(const Problem& pr, const Smem& s) {
  const int words = pr.crit == SLM_MSE ? kPG * pr.B : kPG * pr.B * pr.K;
  for (int i = threadIdx.x; i < words; i += kThreads) s.hist[i] = 0u;
  if (pr.crit == SLM_MSE)
    for (int i = threadIdx.x; i < kPG * pr.B; i += kThreads) {
      s.hs[i] = 0.0;
      s.hq[i] = 0.0;
    }
}

// Sets zmin / inv_w / ok of each particle from s.smin / s.smax.
__device__ __forceinline__ void finish_range(const Problem& pr, const Smem& s) {
  for (int p = threadIdx.x; p < kPG; p += kThreads) {
    if (s.smin[p] == INT_MAX) {  // empty node
      s.ok[p] = 0;
      s.zmin[p] = 0.f;
      s.inv_w[p] = 0.f;
      continue;
    }
    const float lo = ord2f(s.smin[p]), hi = ord2f(s.smax[p]);
    const float width = __fsub_rn(hi, lo);
    const float inv_w = __fdiv_rn((float)pr.B, width);
    s.zmin[p] = lo;
    s.inv_w[p] = inv_w;
    s.ok[p] = (hi > lo) && isfinite(inv_w);
  }
}

// Scans the group's particles (warp w takes particles w, w+8) and writes
// their scores.
__device__ __forceinline__ void scan_group(const Problem& pr, const Smem& s,
                                           EvalRes* out, int p_base) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int pl = warp; pl < kPG; pl += kThreads / 32) {
    if (p_base + pl >= pr.P) continue;
    EvalRes r;
    if (!s.ok[pl]) {
      r = invalid_res();
    } else if (pr.crit == SLM_MSE) {
      r = scan_mse(s.hist + pl * pr.B, s.hs + pl * pr.B, s.hq + pl * pr.B,
                   pr.B, pr.min_leaf);
    } else {
      r = scan_cls(s.hist + (size_t)pl * pr.B * pr.K, pr.B, pr.K, pr.min_leaf,
                   pr.crit);
    }
    r.zmin = s.zmin[pl];
    r.inv_w = s.ok[pl] ? s.inv_w[pl] : 0.f;
    if (lane == 0) out[p_base + pl] = r;
  }
}

// ---- kernels ---------------------------------------------------------------------

// One CTA = one node with <= kSmallMax entries x one particle group.
__global__ void __launch_bounds__(kThreads)
    k_eval_small(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes,
                 const int32_t* __restrict__ list, int32_t* bins_out,
                 int64_t n_idx) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Smem s = carve(smem, pr.crit, pr.B, pr.K);
  const int a = list ? list[blockIdx.x] : blockIdx.x;
  const int g = blockIdx.y;
  const NodeDesc nd = nodes[a];
  const int p_base = g * kPG;
  const float* pos = sw.pos + ((int64_t)a * pr.Pp + p_base) * pr.d;

  for (int p = threadIdx.x; p < kPG; p += kThreads) {
    s.smin[p] = INT_MAX;
    s.smax[p] = INT_MIN;
  }
  float acc[4][4];
  for (int t0 = 0; t0 < nd.seg_len; t0 += kTS) {
    const int n = min(kTS, nd.seg_len - t0);
    __syncthreads();
    load_tile_meta(pr, s, (int64_t)nd.seg_start + t0, n);
    project_tile(pr, s, pos, n, acc);
    tile_minmax(s, n, acc);
  }
  __syncthreads();
  finish_range(pr, s);
  zero_hist(pr, s);
  __syncthreads();
  for (int t0 = 0; t0 < nd.seg_len; t0 += kTS) {
    const int n = min(kTS, nd.seg_len - t0);
    __syncthreads();
    load_tile_meta(pr, s, (int64_t)nd.seg_start + t0, n);
    project_tile(pr, s, pos, n, acc);
    tile_hist(pr, s, n, p_base, acc, bins_out, n_idx, t0);
  }
  __syncthreads();
  scan_group(pr, s, sw.cur + (int64_t)a * pr.Pp, p_base);
}

// Range pass of one work item of a large node.
__global__ void __launch_bounds__(kThreads)
    k_minmax_chunk(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes,
                   const ChunkItem* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Smem s = carve(smem, pr.crit, pr.B, pr.K);
  const ChunkItem it = items[blockIdx.x];
  const int g = blockIdx.y;
  const NodeDesc nd = nodes[it.node];
  const int p_base = g * kPG;
  const float* pos = sw.pos + ((int64_t)it.node * pr.Pp + p_base) * pr.d;
  for (int p = threadIdx.x; p < kPG; p += kThreads) {
    s.smin[p] = INT_MAX;
    s.smax[p] = INT_MIN;
  }
  float acc[4][4];
  for (int t0 = 0; t0 < it.len; t0 += kTS) {
    const int n = min(kTS, it.len - t0);
    __syncthreads();
    load_tile_meta(pr, s, (int64_t)nd.seg_start + it.start + t0, n);
    project_tile(pr, s, pos, n, acc);
    tile_minmax(s, n, acc);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < kPG; p += kThreads) {
    if (s.smin[p] == INT_MAX) continue;
    int* z = sw.zmm + ((int64_t)it.node * pr.Pp + p_base + p) * 2;
    atomicMin(z, s.smin[p]);
    atomicMax(z + 1, s.smax[p]);
  }
}

// Histogram pass of one work item: dense partial histogram to global.
__global__ void __launch_bounds__(kThreads)
    k_hist_chunk(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes,
                 const ChunkItem* __restrict__ items, int32_t* bins_out,
                 int64_t n_idx) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Smem s = carve(smem, pr.crit, pr.B, pr.K);
  const ChunkItem it = items[blockIdx.x];
  const int g = blockIdx.y;
  const NodeDesc nd = nodes[it.node];
  const int p_base = g * kPG;
  const float* pos = sw.pos + ((int64_t)it.node * pr.Pp + p_base) * pr.d;
  for (int p = threadIdx.x; p < kPG; p += kThreads) {
    const int* z = sw.zmm + ((int64_t)it.node * pr.Pp + p_base + p) * 2;
    s.smin[p] = z[0];
    s.smax[p] = z[1];
  }
  __syncthreads();
  finish_range(pr, s);
  zero_hist(pr, s);
  float acc[4][4];
  for (int t0 = 0; t0 < it.len; t0 += kTS) {
    const int n = min(kTS, it.len - t0);
    __syncthreads();
    load_tile_meta(pr, s, (int64_t)nd.seg_start + it.start + t0, n);
    project_tile(pr, s, pos, n, acc);
    tile_hist(pr, s, n, p_base, acc, bins_out, n_idx, it.start + t0);
  }
  __syncthreads();
  // dense copy-out: partial of (item, particle) at ((item*Pp + p) * words)
  const int64_t item = blockIdx.x;
  if (pr.crit == SLM_MSE) {
    const int words = kPG * pr.B;
    const int64_t off = (item * pr.Pp + p_base) * pr.B;
    for (int i = threadIdx.x; i < words; i += kThreads) {
      sw.part[off + i] = s.hist[i];
      sw.part_s[off + i] = s.hs[i];
      sw.part_q[off + i] = s.hq[i];
    }
  } else {
    const int words = kPG * pr.B * pr.K;
    const int64_t off = (item * pr.Pp + p_base) * (int64_t)pr.B * pr.K;
    const uint4* src = reinterpret_cast<const uint4*>(s.hist);
    uint4* dst = reinterpret_cast<uint4*>(sw.part + off);
    if ((words & 3) == 0 && (off & 3) == 0) {
      for (int i = threadIdx.x; i < words / 4; i += kThreads) dst[i] = src[i];
    } else {
      for (int i = threadIdx.x; i < words; i += kThreads)
        sw.part[off + i] = s.hist[i];
    }
  }
}

// One CTA per (large node, particle): sums the item partials and scans.
__global__ void __launch_bounds__(kThreads)
    k_reduce_scan(Problem pr, Swarm sw, const BigNode* __restrict__ big) {
  extern __shared__ __align__(16) unsigned char smem[];
  const BigNode bn = big[blockIdx.x];
  const int p = blockIdx.y;
  if (p >= pr.P) return;
  const int a = bn.node;
  const int B = pr.B;
  const int words = pr.crit == SLM_MSE ? B : B * pr.K;
  uint32_t* h = reinterpret_cast<uint32_t*>(smem);
  double* hs = reinterpret_cast<double*>(smem + ((words * 4 + 15) & ~15));
  double* hq = hs + B;
  for (int i = threadIdx.x; i < words; i += kThreads) {
    uint32_t acc = 0;
    double as = 0.0, aq = 0.0;
    for (int it = 0; it < bn.n_items; ++it) {
      const int64_t off = ((int64_t)(bn.item0 + it) * pr.Pp + p) * words + i;
      acc += sw.part[off];
      if (pr.crit == SLM_MSE) {
        as += sw.part_s[off];
        aq += sw.part_q[off];
      }
    }
    h[i] = acc;
    if (pr.crit == SLM_MSE) {
      hs[i] = as;
      hq[i] = aq;
    }
  }
  __shared__ float s_zmin, s_inv_w;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int* z = sw.zmm + ((int64_t)a * pr.Pp + p) * 2;
    const int lo_o = z[0], hi_o = z[1];
    z[0] = INT_MAX;  // reset for the next iteration
    z[1] = INT_MIN;
    if (lo_o == INT_MAX) {
      s_ok = 0;
      s_zmin = 0.f;
      s_inv_w = 0.f;
    } else {
      const float lo = ord2f(lo_o), hi = ord2f(hi_o);
      const float inv_w = __fdiv_rn((float)B, __fsub_rn(hi, lo));
      s_zmin = lo;
      s_inv_w = inv_w;
      s_ok = (hi > lo) && isfinite(inv_w);
    }
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  EvalRes r;
  if (!s_ok)
    r = invalid_res();
  else if (pr.crit == SLM_MSE)
    r = scan_mse(h, hs, hq, B, pr.min_leaf);
  else
    r = scan_cls(h, B, pr.K, pr.min_leaf, pr.crit);
  r.zmin = s_zmin;
  r.inv_w = s_ok ? s_inv_w : 0.f;
  if (threadIdx.x == 0) sw.cur[(int64_t)a * pr.Pp + p] = r;
}

// Initial swarm of each node: x ~ U[-1,1)^d, v ~ 0.1 U[-1,1)^d.
__global__ void k_swarm_init(Problem pr, Swarm sw,
                             const NodeDesc* __restrict__ nodes,
                             SwarmCoef co) {
  const int a = blockIdx.x;
  const uint32_t uid = nodes[a].uid;
  const int d = pr.d, d4 = (d + 3) >> 2;
  const uint32_t k0 = (uint32_t)co.seed, k1 = (uint32_t)(co.seed >> 32);
  float* pos = sw.pos + (int64_t)a * pr.Pp * d;
  float* vel = sw.vel + (int64_t)a * pr.Pp * d;
  for (int e = threadIdx.x; e < pr.Pp * d4; e += blockDim.x) {
    const int p = e / d4, q = e - p * d4;
    if (p >= pr.P) {
      for (int c = 0; c < 4; ++c) {
        const int j = 4 * q + c;
        if (j < d) {
          pos[(int64_t)p * d + j] = 0.f;
          vel[(int64_t)p * d + j] = 0.f;
        }
      }
      continue;
    }
    const U4 rx = philox4x32_10(uid, 0u, (uint32_t)p,
                                (uint32_t)q | (kInitX << 24), k0, k1);
    const U4 rv = philox4x32_10(uid, 0u, (uint32_t)p,
                                (uint32_t)q | (kInitV << 24), k0, k1);
    for (int c = 0; c < 4; ++c) {
      const int j = 4 * q + c;
      if (j >= d) break;
      const float ux = uniform24(rx.v[c]), uv = uniform24(rv.v[c]);
      pos[(int64_t)p * d + j] = __fsub_rn(__fmul_rn(2.0f, ux), 1.0f);
      vel[(int64_t)p * d + j] =
          __fmul_rn(0.1f, __fsub_rn(__fmul_rn(2.0f, uv), 1.0f));
    }
  }
  for (int p = threadIdx.x; p < pr.Pp; p += blockDim.x) {
    int* z = sw.zmm + ((int64_t)a * pr.Pp + p) * 2;
    z[0] = INT_MAX;
    z[1] = INT_MIN;
  }
  if (threadIdx.x == 0) {
    sw.gb[a] = invalid_res();
    sw.gpart[a] = 0;
    sw.giter[a] = 0;
  }
}

// Bests after evaluation t (Algorithm 1, strict "<", particles in increasing
// order), then -- if t < T -- the synchronous move to iteration t+1.
__global__ void __launch_bounds__(kThreads)
    k_swarm_update(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes,
                   int t, SwarmCoef co) {
  const int a = blockIdx.x;
  const int P = pr.P, Pp = pr.Pp, d = pr.d;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ int s_imp[kMaxParticles];
  __shared__ EvalRes s_wbest[kThreads / 32];
  __shared__ int s_widx[kThreads / 32];
  __shared__ int s_best;
  EvalRes* cur = sw.cur + (int64_t)a * Pp;
  EvalRes* pb = sw.pb + (int64_t)a * Pp;
  const EvalRes gold = sw.gb[a];

  // pbest scores; gbest candidates = particles strictly better than gold
  // (at t = 0 every particle; gold is then unset).
  const int p = threadIdx.x;
  EvalRes ce = invalid_res();
  int cidx = INT_MAX;
  if (p < P) {
    ce = cur[p];
    const bool imp = (t == 0) || better(ce, pb[p], pr.crit);
    s_imp[p] = imp;
    if (imp) pb[p] = ce;
    if (t == 0 || better(ce, gold, pr.crit)) cidx = p;
  }
  // argmin over candidates: better score, ties to the lower index
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const EvalRes o = shfl_res(ce, lane ^ off);
    const int oi = __shfl_xor_sync(0xffffffffu, cidx, off);
    bool take;
    if (oi == INT_MAX)
      take = false;
    else if (cidx == INT_MAX)
      take = true;
    else if (better(o, ce, pr.crit))
      take = true;
    else if (better(ce, o, pr.crit))
      take = false;
    else
      take = oi < cidx;
    if (take) {
      ce = o;
      cidx = oi;
    }
  }
  if (lane == 0) {
    s_wbest[warp] = ce;
    s_widx[warp] = cidx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    EvalRes b = s_wbest[0];
    int bi = s_widx[0];
    for (int w = 1; w < kThreads / 32; ++w) {
      const EvalRes o = s_wbest[w];
      const int oi = s_widx[w];
      if (oi == INT_MAX) continue;
      if (bi == INT_MAX || better(o, b, pr.crit) ||
          (!better(b, o, pr.crit) && oi < bi)) {
        b = o;
        bi = oi;
      }
    }
    s_best = bi == INT_MAX ? -1 : bi;
    if (bi != INT_MAX) {
      sw.gb[a] = b;
      sw.gpart[a] = bi;
      sw.giter[a] = t;
    }
    if (sw.trace) {
      const EvalRes g = bi != INT_MAX ? b : gold;
      sw.trace[(int64_t)a * (sw.T + 1) + t] =
          g.valid ? g.loss : __longlong_as_double(0x7ff0000000000000LL);
    }
  }
  __syncthreads();
  float* pos = sw.pos + (int64_t)a * Pp * d;
  float* vel = sw.vel + (int64_t)a * Pp * d;
  float* pbp = sw.pbest + (int64_t)a * Pp * d;
  float* gbp = sw.gbest + (int64_t)a * d;
  const int best = s_best;
  for (int e = threadIdx.x; e < P * d; e += kThreads) {
    const int q = e / d;
    if (s_imp[q]) pbp[e] = pos[e];
  }
  if (best >= 0)
    for (int j = threadIdx.x; j < d; j += kThreads)
      gbp[j] = pos[(int64_t)best * d + j];
  if (t >= sw.T) return;
  __syncthreads();

  // v <- omega v + (c1 r1)(pB - x) + (c2 r2)(gB - x);  x <- x + v
  const uint32_t uid = nodes[a].uid;
  const uint32_t k0 = (uint32_t)co.seed, k1 = (uint32_t)(co.seed >> 32);
  const int d4 = (d + 3) >> 2;
  for (int e = threadIdx.x; e < P * d4; e += kThreads) {
    const int pi = e / d4, q = e - pi * d4;
    const U4 r1 = philox4x32_10(uid, (uint32_t)(t + 1), (uint32_t)pi,
                                (uint32_t)q | (kR1 << 24), k0, k1);
    const U4 r2 = philox4x32_10(uid, (uint32_t)(t + 1), (uint32_t)pi,
                                (uint32_t)q | (kR2 << 24), k0, k1);
    for (int c = 0; c < 4; ++c) {
      const int j = 4 * q + c;
      if (j >= d) break;
      const int64_t ix = (int64_t)pi * d + j;
      const float x = pos[ix], v = vel[ix];
      const float inertia = __fmul_rn(co.inertia, v);
      const float cog = __fmul_rn(__fmul_rn(co.c1, uniform24(r1.v[c])),
                                  __fsub_rn(pbp[ix], x));
      const float soc = __fmul_rn(__fmul_rn(co.c2, uniform24(r2.v[c])),
                                  __fsub_rn(gbp[j], x));
      const float vn = __fadd_rn(__fadd_rn(inertia, cog), soc);
      vel[ix] = vn;
      pos[ix] = __fadd_rn(x, vn);
    }
  }
}

__global__ void k_swarm_uniforms(uint64_t seed, uint32_t uid, uint32_t t,
                                 int P, int d, uint32_t purpose, float* u) {
  const int d4 = (d + 3) >> 2;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)P * d4) return;
  const int p = (int)(e / d4), q = (int)(e - (int64_t)p * d4);
  const U4 r = philox4x32_10(uid, t, (uint32_t)p, (uint32_t)q | (purpose << 24),
                             (uint32_t)seed, (uint32_t)(seed >> 32));
  for (int c = 0; c < 4; ++c) {
    const int j = 4 * q + c;
    if (j < d) u[(int64_t)p * d + j] = uniform24(r.v[c]);
  }
}

__global__ void k_bootstrap(uint64_t seed, uint32_t tree, int64_t n,
                            uint32_t* w) {
  const int64_t blk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blk * 4 >= n) return;
  const U4 r = philox4x32_10(tree, (uint32_t)blk, 0u, kBootstrap << 24,
                             (uint32_t)seed, (uint32_t)(seed >> 32));
  for (int c = 0; c < 4; ++c) {
    const int64_t k = blk * 4 + c;
    if (k >= n) break;
    const uint64_t s = ((uint64_t)r.v[c] * (uint64_t)n) >> 32;
    atomicAdd(&w[s], 1u);
  }
}

}  // namespace

// ---- launchers ---------------------------------------------------------------------

size_t eval_smem_bytes(const Problem& pr) {
  return hist_bytes(pr.crit, pr.B, pr.K) + 16 + fixed_bytes();
}

static size_t reduce_smem_bytes(const Problem& pr) {
  const int words = pr.crit == SLM_MSE ? pr.B : pr.B * pr.K;
  return ((words * 4 + 15) & ~15) + (pr.crit == SLM_MSE ? 16 * pr.B : 0);
}

cudaError_t prepare_eval_kernels(const Problem& pr) {
  const int bytes = (int)eval_smem_bytes(pr);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_eval_small,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes)))
    return e;
  if ((e = cudaFuncSetAttribute(k_minmax_chunk,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes)))
    return e;
  if ((e = cudaFuncSetAttribute(k_hist_chunk,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes)))
    return e;
  return cudaFuncSetAttribute(k_reduce_scan,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)reduce_smem_bytes(pr));
}

cudaError_t launch_swarm_init(const Problem& pr, const Swarm& sw,
                              const NodeDesc* nodes, int A, SwarmCoef co,
                              cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  k_swarm_init<<<A, kThreads, 0, st>>>(pr, sw, nodes, co);
  return cudaGetLastError();
}

cudaError_t launch_eval_small(const Problem& pr, const Swarm& sw,
                              const NodeDesc* nodes, const int32_t* list,
                              int n_list, cudaStream_t st) {
  if (n_list <= 0) return cudaSuccess;
  dim3 grid(n_list, pr.G);
  k_eval_small<<<grid, kThreads, eval_smem_bytes(pr), st>>>(pr, sw, nodes, list,
                                                            nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_minmax_chunk(const Problem& pr, const Swarm& sw,
                                const NodeDesc* nodes, const ChunkItem* items,
                                int n_items, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  k_minmax_chunk<<<dim3(n_items, pr.G), kThreads, eval_smem_bytes(pr), st>>>(
      pr, sw, nodes, items);
  return cudaGetLastError();
}

cudaError_t launch_hist_chunk(const Problem& pr, const Swarm& sw,
                              const NodeDesc* nodes, const ChunkItem* items,
                              int n_items, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  k_hist_chunk<<<dim3(n_items, pr.G), kThreads, eval_smem_bytes(pr), st>>>(
      pr, sw, nodes, items, nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_reduce_scan(const Problem& pr, const Swarm& sw,
                               const BigNode* big, int n_big, cudaStream_t st) {
  if (n_big <= 0) return cudaSuccess;
  k_reduce_scan<<<dim3(n_big, pr.P), kThreads, reduce_smem_bytes(pr), st>>>(
      pr, sw, big);
  return cudaGetLastError();
}

cudaError_t launch_eval_positions(const Problem& pr, const Swarm& sw,
                                  const NodeDesc* node, const ChunkItem* items,
                                  int n_items, const BigNode* big,
                                  int32_t* bins_out, int64_t n_idx,
                                  cudaStream_t st) {
  const size_t sm = eval_smem_bytes(pr);
  if (n_items == 0) {
    k_eval_small<<<dim3(1, pr.G), kThreads, sm, st>>>(pr, sw, node, nullptr,
                                                      bins_out, n_idx);
    return cudaGetLastError();
  }
  dim3 grid(n_items, pr.G);
  k_minmax_chunk<<<grid, kThreads, sm, st>>>(pr, sw, node, items);
  k_hist_chunk<<<grid, kThreads, sm, st>>>(pr, sw, node, items, bins_out, n_idx);
  k_reduce_scan<<<dim3(1, pr.P), kThreads, reduce_smem_bytes(pr), st>>>(pr, sw,
                                                                        big);
  return cudaGetLastError();
}

cudaError_t launch_swarm_update(const Problem& pr, const Swarm& sw,
                                const NodeDesc* nodes, int A, int t,
                                SwarmCoef co, cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  k_swarm_update<<<A, kThreads, 0, st>>>(pr, sw, nodes, t, co);
  return cudaGetLastError();
}

cudaError_t launch_swarm_uniforms(uint64_t seed, uint32_t uid, uint32_t t,
                                  int P, int d, uint32_t purpose, float* u,
                                  cudaStream_t st) {
  const int64_t n = (int64_t)P * ((d + 3) / 4);
  if (n <= 0) return cudaSuccess;
  k_swarm_uniforms<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(seed, uid, t, P,
                                                                d, purpose, u);
  return cudaGetLastError();
}

cudaError_t launch_bootstrap(uint64_t seed, uint32_t tree, int64_t n,
                             uint32_t* w, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(w, 0, sizeof(uint32_t) * n, st);
  if (e) return e;
  const int64_t blocks = (n + 4 * 256 - 1) / (4 * 256);
  if (blocks > 0) k_bootstrap<<<(unsigned)blocks, 256, 0, st>>>(seed, tree, n, w);
  return cudaGetLastError();
}

}  // namespace slm
