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
// Data layout. A batch's rows are stored entry-ordered and contiguous (the
// level-resident copy X_l[E, d]: each node is a segment of consecutive rows),
// with entry-aligned labels / targets / multiplicities. One iteration is two
// kernels plus the swarm update:
//  * k_project: z[p][e] = X_l[e] . x_p for all entries and particles, once.
//    A persistent grid walks (tile of kTS = 256 rows, group of kPG = 16
//    particles) work units; rows and positions stream through shared memory
//    in kKC = 32-feature chunks with double-buffered cp.async copies. Each
//    thread owns a 4 x 4 register tile (rows w*32 + sg + 8i, particles
//    pg + 4j) and accumulates over the features in increasing order, so every
//    z is the same sequence of fused multiply-adds whatever the tiling. The
//    per-(node, particle) range is folded in with ordered-int atomics and z is
//    written to an L2-resident buffer.
//  * k_hist_scan: one CTA per (node, particle) bins the node's z into
//    warp-private shared histograms, merges them and scans the edges.
#include <cuda_runtime.h>
#include <float.h>
#include <limits.h>
#include <math.h>

#include <cooperative_groups.h>

#include "philox.cuh"
#include "slm_internal.cuh"

namespace slm {

namespace {

// ---- small helpers -----------------------------------------------------------

// Programmatic dependent launch: the next kernel of the stream may begin
// launching once every CTA of this grid has passed pdl_trigger(); pdl_wait()
// blocks until the previous grid has completed and its writes are visible.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

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
  uint32_t occ[kMaxBPL];  // samples in bin j0 + i (all classes)
#pragma unroll
  for (int i = 0; i < kMaxBPL; ++i) occ[i] = 0;
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
      occ[i] += c[i];
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
    if (occ[i] == 0) continue;  // same partition as edge b-1
    const uint32_t nl = nL[i], nr = ntot - nl;
    if (nl < (uint32_t)min_leaf || nr < (uint32_t)min_leaf) continue;
    EvalRes c = invalid_res();
    c.valid = 1;
    c.bin = b;
    c.nl = nl;
    c.nr = nr;
    if (crit == SLM_GINI) {
      // decisions use the exact rational; the double loss is formed once, for
      // the winning edge (FP64 division is slow on this part)
      c.num = SL[i] * nr + SR[i] * nl;
      c.den = (uint64_t)nl * nr;
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
  if (crit == SLM_GINI && best.valid) {
    const uint64_t nden = (uint64_t)ntot * best.den;
    best.loss = (double)(nden - best.num) / (double)nden;
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
    // an empty bin b-1 gives edge b the partition of edge b-1: keep the lower
    if (c[i] == 0) continue;
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

// ---- async copies -------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src),
               "r"(bytes));
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(src),
               "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::);
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// ---- bulk copies (TMA) with mbarrier completion -------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// 1D bulk copy global -> this CTA's shared memory; 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Waits for phase `parity` of the barrier, at most `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
  const uint32_t a = smem_addr(bar);
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
constexpr int kWaitPolls = 1 << 20;  // bounded: a lost copy ends the kernel, not the GPU

// ---- projection -------------------------------------------------------------------

constexpr size_t kProjSmem = sizeof(float) * 2 * (kTS * kXS + kPG * kXS);

// Stages one kKC-feature chunk of a work unit's rows and positions.
__device__ __forceinline__ void stage_chunk(const Problem& pr, const Swarm& sw,
                                            const WorkTile& wt, int g, int k0,
                                            bool vec, float* xb, float* ab) {
  const int d = pr.d;
  const int kc = min(kKC, d - k0);
  const float* pos = sw.pos + ((int64_t)wt.node * pr.Pp + g * kPG) * d;
  if (vec) {
    for (int q = threadIdx.x; q < kTS * (kKC / 4); q += kThreads) {
      const int r = q >> 3, cc = (q & 7) * 4;
      const bool ok = r < wt.rows && cc < kc;
      const float* src = ok ? pr.X + (int64_t)(wt.row0 + r) * d + k0 + cc : pr.X;
      cp_async16(xb + r * kXS + cc, src, ok ? 16 : 0);
    }
    for (int q = threadIdx.x; q < kPG * (kKC / 4); q += kThreads) {
      const int p = q >> 3, cc = (q & 7) * 4;
      const bool ok = cc < kc;
      cp_async16(ab + p * kXS + cc, ok ? pos + (int64_t)p * d + k0 + cc : pos, ok ? 16 : 0);
    }
  } else {
    for (int q = threadIdx.x; q < kTS * kKC; q += kThreads) {
      const int r = q >> 5, cc = q & 31;
      const bool ok = r < wt.rows && cc < kc;
      const float* src = ok ? pr.X + (int64_t)(wt.row0 + r) * d + k0 + cc : pr.X;
      cp_async4(xb + r * kXS + cc, src, ok ? 4 : 0);
    }
    for (int q = threadIdx.x; q < kPG * kKC; q += kThreads) {
      const int p = q >> 5, cc = q & 31;
      const bool ok = cc < kc;
      cp_async4(ab + p * kXS + cc, ok ? pos + (int64_t)p * d + k0 + cc : pos, ok ? 4 : 0);
    }
  }
  cp_async_commit();
}

__global__ void __launch_bounds__(kThreads, 2)
    k_project(Problem pr, Swarm sw, const WorkTile* __restrict__ tiles, int n_units) {
  extern __shared__ __align__(16) float smf[];
  float* xs0 = smf;
  float* xs1 = smf + kTS * kXS;
  float* as0 = smf + 2 * kTS * kXS;
  float* as1 = as0 + kPG * kXS;
  pdl_trigger();
  pdl_wait();
  if ((int)blockIdx.x >= n_units) return;
  const int d = pr.d, G = pr.G;
  const int nk = (d + kKC - 1) / kKC;
  const bool vec = (d & 3) == 0;
  const int my_units = (n_units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;
  const int n_st = my_units * nk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sg = lane & 7, pg = lane >> 3;

  {
    const int u = blockIdx.x;
    stage_chunk(pr, sw, tiles[u / G], u % G, 0, vec, xs0, as0);
  }
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;

  for (int s = 0; s < n_st; ++s) {
    const int ui = s / nk, c = s - ui * nk;
    const int u = blockIdx.x + ui * gridDim.x;
    if (s + 1 < n_st) {
      const int ui1 = (s + 1) / nk, c1 = (s + 1) - ui1 * nk;
      const int u1 = blockIdx.x + ui1 * gridDim.x;
      stage_chunk(pr, sw, tiles[u1 / G], u1 % G, c1 * kKC, vec, (s & 1) ? xs0 : xs1,
                  (s & 1) ? as0 : as1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* xb = (s & 1) ? xs1 : xs0;
    const float* ab = (s & 1) ? as1 : as0;
    const int kc4 = (min(kKC, d - c * kKC) + 3) & ~3;
    const float* xr = xb + (warp * 32 + sg) * kXS;
    const float* ar = ab + pg * kXS;
#pragma unroll 2
    for (int k = 0; k < kc4; k += 4) {
      float4 xv[4], av[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xv[i] = *reinterpret_cast<const float4*>(xr + i * 8 * kXS + k);
#pragma unroll
      for (int j = 0; j < 4; ++j) av[j] = *reinterpret_cast<const float4*>(ar + j * 4 * kXS + k);
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
    if (c == nk - 1) {
      // tile complete: fold the range, store z
      const WorkTile wt = tiles[u / G];
      const int g = u % G;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int p = g * kPG + pg + 4 * j;
        float lo = FLT_MAX, hi = -FLT_MAX;
        bool any = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = warp * 32 + sg + 8 * i;
          if (r < wt.rows) {
            const float z = acc[i][j];
            lo = z < lo ? z : lo;
            hi = z > hi ? z : hi;
            any = true;
            if (p < pr.P) sw.z[(int64_t)p * pr.Ez + wt.row0 + r] = z;
          }
        }
        int olo = any ? f2ord(lo) : INT_MAX, ohi = any ? f2ord(hi) : INT_MIN;
#pragma unroll
        for (int off = 1; off < 8; off <<= 1) {
          olo = min(olo, __shfl_xor_sync(0xffffffffu, olo, off));
          ohi = max(ohi, __shfl_xor_sync(0xffffffffu, ohi, off));
        }
        if (sg == 0 && olo != INT_MAX && p < pr.P) {
          int* zz = sw.zmm + ((int64_t)wt.node * pr.Pp + p) * 2;
          atomicMin(zz, olo);
          atomicMax(zz + 1, ohi);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    }
    __syncthreads();  // buffer s&1 is refilled by the next stage's copies
  }
}

// ---- swarm update ----------------------------------------------------------------

__device__ __forceinline__ EvalRes ldcg_res(const EvalRes* p) {
  EvalRes r;
  r.loss = __ldcg(&p->loss);
  r.num = __ldcg((const unsigned long long*)&p->num);
  r.den = __ldcg((const unsigned long long*)&p->den);
  r.zmin = __ldcg(&p->zmin);
  r.inv_w = __ldcg(&p->inv_w);
  r.bin = __ldcg(&p->bin);
  r.valid = __ldcg(&p->valid);
  r.nl = __ldcg((const long long*)&p->nl);
  r.nr = __ldcg((const long long*)&p->nr);
  return r;
}

// Algorithm 1, pbest step of particle p after evaluation t (one warp): strict
// "<" against the particle's best so far; the position is kept on improvement.
__device__ __forceinline__ void pbest_step(const Problem& pr, const Swarm& sw, int a, int p,
                                           int t, const EvalRes& cur) {
  const int lane = threadIdx.x & 31;
  EvalRes* pb = sw.pb + (int64_t)a * pr.Pp + p;
  int imp = 0;
  if (lane == 0) {
    imp = (t == 0) || better(cur, *pb, pr.crit);
    if (imp) *pb = cur;
  }
  imp = __shfl_sync(0xffffffffu, imp, 0);
  if (!imp) return;
  const int64_t o = ((int64_t)a * pr.Pp + p) * pr.d;
  for (int j = lane; j < pr.d; j += 32) sw.pbest[o + j] = sw.pos[o + j];
}

// Algorithm 1, gbest step of node a after evaluation t. Run by all threads of
// the CTA that finished the node's last particle group in this iteration.
__device__ void node_tail(const Problem& pr, const Swarm& sw, int a, int t) {
  const int P = pr.P, Pp = pr.Pp, d = pr.d;
  const int nthr = blockDim.x, nw = nthr >> 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ EvalRes s_wbest[kThreads / 32];
  __shared__ int s_widx[kThreads / 32];
  __shared__ int s_best;
  const EvalRes* cur = sw.cur + (int64_t)a * Pp;
  const EvalRes gold = sw.gb[a];

  // gbest candidates = particles strictly better than gold (at t = 0 every
  // particle; gold is then unset); argmin with ties to the lower index
  EvalRes ce = invalid_res();
  int cidx = INT_MAX;
  for (int p = threadIdx.x; p < P; p += nthr) {
    const EvalRes e = ldcg_res(cur + p);  // written by other CTAs of this launch
    if (!(t == 0 || better(e, gold, pr.crit))) continue;
    if (cidx == INT_MAX || better(e, ce, pr.crit)) {
      ce = e;
      cidx = p;
    }
  }
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
    for (int w = 1; w < nw; ++w) {
      const EvalRes o = s_wbest[w];
      const int oi = s_widx[w];
      if (oi == INT_MAX) continue;
      if (bi == INT_MAX || better(o, b, pr.crit) || (!better(b, o, pr.crit) && oi < bi)) {
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
  // the new gbest improved its pbest in this iteration, so its pbest row is
  // its current position (written by another CTA of this launch)
  const float* pbp = sw.pbest + (int64_t)a * Pp * d;
  float* gbp = sw.gbest + (int64_t)a * d;
  const int best = s_best;
  if (best >= 0)
    for (int j = threadIdx.x; j < d; j += nthr) gbp[j] = __ldcg(pbp + (int64_t)best * d + j);
}

// Eq. pso-1, synchronous: every particle moves with the gbest held at the end
// of iteration t. One thread per (node, particle, 4 dimensions).
__global__ void __launch_bounds__(128)
    k_move(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes, int A, int t,
           SwarmCoef co) {
  pdl_trigger();
  pdl_wait();
  const int d = pr.d, d4 = (d + 3) >> 2;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per_node = (int64_t)pr.P * d4;
  if (item >= per_node * A) return;
  const int a = (int)(item / per_node);
  const int rem = (int)(item - (int64_t)a * per_node);
  const int pi = rem / d4, q = rem - pi * d4;
  const uint32_t uid = nodes[a].uid;
  const uint32_t k0 = (uint32_t)co.seed, k1 = (uint32_t)(co.seed >> 32);
  const U4 r1 = philox4x32_10(uid, (uint32_t)(t + 1), (uint32_t)pi, (uint32_t)q | (kR1 << 24),
                              k0, k1);
  const U4 r2 = philox4x32_10(uid, (uint32_t)(t + 1), (uint32_t)pi, (uint32_t)q | (kR2 << 24),
                              k0, k1);
  const int64_t row = ((int64_t)a * pr.Pp + pi) * d;
  float* pos = sw.pos + row;
  float* vel = sw.vel + row;
  const float* pbp = sw.pbest + row;
  const float* gbp = sw.gbest + (int64_t)a * d;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = 4 * q + c;
    if (j >= d) break;
    // v <- omega v + (c1 r1)(pB - x) + (c2 r2)(gB - x);  x <- x + v
    const float x = pos[j], v = vel[j];
    const float inertia = __fmul_rn(co.inertia, v);
    const float cog = __fmul_rn(__fmul_rn(co.c1, uniform24(r1.v[c])), __fsub_rn(pbp[j], x));
    const float soc = __fmul_rn(__fmul_rn(co.c2, uniform24(r2.v[c])), __fsub_rn(gbp[j], x));
    const float vn = __fadd_rn(__fadd_rn(inertia, cog), soc);
    vel[j] = vn;
    pos[j] = __fadd_rn(x, vn);
  }
}

// ---- histogram and scan -------------------------------------------------------------

constexpr int kWP = 8;        // particles per CTA of the histogram kernel, one per warp
constexpr int kPiece = 1024;  // entries per staged piece

__host__ __device__ inline size_t hist_particle_bytes(int crit, int B, int K) {
  return crit == SLM_MSE ? (size_t)B * (4 + 8 + 8) : (size_t)B * K * 4;
}
// One staged piece: z of kWP particles, then labels or targets, then
// multiplicities (if weighted).
__host__ __device__ inline size_t stage_bytes(bool weighted) {
  return (size_t)kPiece * 4 * (kWP + 1 + (weighted ? 1 : 0));
}

// A cluster of S CTAs per (node, group of kWP particles). Warp w of every
// CTA owns particle g*kWP + w. The CTA's slice of the node's entries (rank r:
// the r-th of S slices) streams through shared memory in kPiece-entry pieces:
// one thread issues bulk (TMA) copies of the kWP z rows, the labels / targets
// and the multiplicities of a piece, double-buffered on two mbarriers; every
// warp bins its particle's z from shared memory into its own histogram. Rank
// q of the cluster then sums one slice of every histogram word over the S
// CTAs through distributed shared memory into rank 0, whose warps scan the
// B-1 edges of their particles. In a search (do_update) each warp also takes
// its particle's pbest step, and the CTA that finishes a node's last particle
// group (ticket in sw.done) runs the node's gbest step (the move is k_move).
__global__ void __launch_bounds__(kThreads)
    k_hist_scan(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes, int32_t* bins_out,
                int t, SwarmCoef co, int do_update) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int s_last;
  const cg::cluster_group cl = cg::this_cluster();
  pdl_trigger();
  pdl_wait();
  const int S = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int a = blockIdx.x / S;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = blockIdx.y;
  const int p = g * kWP + warp;
  const bool live = p < pr.P;
  const NodeDesc nd = nodes[a];
  const int B = pr.B, K = pr.K;
  const bool mse = pr.crit == SLM_MSE;
  const bool weighted = pr.w != nullptr;
  const int words = mse ? B : B * K;  // u32 counters per particle
  // shared memory: histograms, then two stages
  double* hs = reinterpret_cast<double*>(smem);         // MSE [kWP][B]
  double* hq = hs + (mse ? kWP * B : 0);                 // MSE [kWP][B]
  uint32_t* hc = reinterpret_cast<uint32_t*>(hq + (mse ? kWP * B : 0));  // [kWP][words]
  unsigned char* stage0 =
      smem + (((size_t)hist_particle_bytes(pr.crit, B, K) * kWP + 127) & ~(size_t)127);
  const size_t sbytes = stage_bytes(weighted);
  uint32_t* h = hc + warp * words;
  double* hsw = hs + warp * B;
  double* hqw = hq + warp * B;

  // range of this warp's particle
  int lo_o = INT_MAX, hi_o = INT_MIN;
  int* zz = sw.zmm + ((int64_t)a * pr.Pp + (live ? p : 0)) * 2;
  if (live && lane == 0) {
    lo_o = zz[0];
    hi_o = zz[1];
  }
  lo_o = __shfl_sync(0xffffffffu, lo_o, 0);
  hi_o = __shfl_sync(0xffffffffu, hi_o, 0);
  float zmin = 0.f, inv_w = 0.f;
  bool ok = false;
  if (lo_o != INT_MAX) {
    const float lo = ord2f(lo_o), hi = ord2f(hi_o);
    inv_w = __fdiv_rn((float)B, __fsub_rn(hi, lo));
    zmin = lo;
    ok = (hi > lo) && isfinite(inv_w);
  }
  for (int i = lane; i < words; i += 32) h[i] = 0u;
  if (mse)
    for (int i = lane; i < B; i += 32) {
      hsw[i] = 0.0;
      hqw[i] = 0.0;
    }
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();

  // slice of this rank: starts on a multiple of 4 entries (16 bytes)
  const int chunk = ((nd.seg_len + S - 1) / S + 3) & ~3;
  const int r_begin = min(nd.seg_len, rank * chunk);
  const int r_end = min(nd.seg_len, r_begin + chunk);
  const int n_pieces = (r_end - r_begin + kPiece - 1) / kPiece;
  const int64_t e0 = nd.seg_start;  // multiple of 4
  const int n_live = min(kWP, pr.P - g * kWP);
  auto issue = [&](int k) {
    const int r = r_begin + k * kPiece;
    const int n = min(kPiece, r_end - r);
    const uint32_t bytes = (uint32_t)(((n + 3) & ~3) * 4);
    unsigned char* st = stage0 + (k & 1) * sbytes;
    uint64_t* bar = &s_bar[k & 1];
    fence_proxy_async();
    mbar_expect_tx(bar, bytes * (uint32_t)(n_live + 1 + (weighted ? 1 : 0)));
    for (int w = 0; w < n_live; ++w)
      bulk_g2s(st + (size_t)w * kPiece * 4, sw.z + (int64_t)(g * kWP + w) * pr.Ez + e0 + r,
               bytes, bar);
    const void* src = mse ? (const void*)(pr.y + e0 + r) : (const void*)(pr.lab + e0 + r);
    bulk_g2s(st + (size_t)kWP * kPiece * 4, src, bytes, bar);
    if (weighted) bulk_g2s(st + (size_t)(kWP + 1) * kPiece * 4, pr.w + e0 + r, bytes, bar);
  };
  if (threadIdx.x == 0 && n_pieces > 0) issue(0);
  bool lost = false;
  for (int k = 0; k < n_pieces; ++k) {
    if (threadIdx.x == 0 && k + 1 < n_pieces) issue(k + 1);
    if (!mbar_wait(&s_bar[k & 1], (uint32_t)((k >> 1) & 1), kWaitPolls)) {
      // a copy did not land: record it, give in-flight copies a bounded
      // chance to finish, and stop using the stages
      if (threadIdx.x == 0 && sw.err) atomicExch(sw.err, 3);
      mbar_wait(&s_bar[k & 1], (uint32_t)((k >> 1) & 1), kWaitPolls);
      if (k + 1 < n_pieces) mbar_wait(&s_bar[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1), kWaitPolls);
      lost = true;
      break;
    }
    const unsigned char* st = stage0 + (k & 1) * sbytes;
    const int r = r_begin + k * kPiece;
    const int n = min(kPiece, r_end - r);
    if (live && ok) {
      const float* zs = reinterpret_cast<const float*>(st) + (size_t)warp * kPiece;
      const int32_t* ls = reinterpret_cast<const int32_t*>(st + (size_t)kWP * kPiece * 4);
      const float* ys = reinterpret_cast<const float*>(st + (size_t)kWP * kPiece * 4);
      const uint32_t* ws =
          reinterpret_cast<const uint32_t*>(st + (size_t)(kWP + 1) * kPiece * 4);
      for (int i = lane; i < n; i += 32) {
        const int b = bin_of(zs[i], zmin, inv_w, B);
        const uint32_t w = weighted ? ws[i] : 1u;
        if (mse) {
          const float yv = ys[i];
          const double wy = (double)w * (double)yv;
          atomicAdd(&h[b], w);
          atomicAdd(&hsw[b], wy);
          atomicAdd(&hqw[b], wy * (double)yv);
        } else {
          atomicAdd(&h[b * K + ls[i]], w);
        }
        if (bins_out) bins_out[(int64_t)p * nd.seg_len + r + i] = b;
      }
    }
    __syncthreads();  // stage k & 1 is refilled by piece k + 2
  }
  (void)lost;
  if (S > 1) {
    cl.sync();  // every CTA's histograms are complete
    // rank q sums words [q*W/S, (q+1)*W/S) of all kWP histograms into rank 0
    const int W = kWP * words;
    const int w0 = (int)((int64_t)W * rank / S), w1 = (int)((int64_t)W * (rank + 1) / S);
    uint32_t* dst = cl.map_shared_rank(hc, 0);
    for (int i = w0 + threadIdx.x; i < w1; i += kThreads) {
      uint32_t v = 0;
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (q < S) v += cl.map_shared_rank(hc, q)[i];
      dst[i] = v;
    }
    if (mse) {
      const int Wd = kWP * B;
      const int d0 = (int)((int64_t)Wd * rank / S), d1 = (int)((int64_t)Wd * (rank + 1) / S);
      double* ds = cl.map_shared_rank(hs, 0);
      double* dq = cl.map_shared_rank(hq, 0);
      for (int i = d0 + threadIdx.x; i < d1; i += kThreads) {
        double vs = 0.0, vq = 0.0;
        for (int q = 0; q < S; ++q) {
          vs += cl.map_shared_rank(hs, q)[i];
          vq += cl.map_shared_rank(hq, q)[i];
        }
        ds[i] = vs;
        dq[i] = vq;
      }
    }
    cl.sync();  // rank 0 holds the sums; the others' memory is no longer read
    if (rank != 0) return;
  }
  if (live) {
    if (lane == 0) {
      zz[0] = INT_MAX;  // ready for the next iteration
      zz[1] = INT_MIN;
    }
    EvalRes res;
    if (!ok) {
      res = invalid_res();
    } else {
      res = mse ? scan_mse(h, hsw, hqw, B, pr.min_leaf) : scan_cls(h, B, K, pr.min_leaf, pr.crit);
      res.zmin = zmin;
      res.inv_w = inv_w;
    }
    if (lane == 0) sw.cur[(int64_t)a * pr.Pp + p] = res;
    if (do_update) pbest_step(pr, sw, a, p, t, res);
  }
  if (!do_update) return;
  __threadfence();  // this CTA's scores and pbest rows, before its ticket
  __syncthreads();
  if (threadIdx.x == 0) {
    const int prev = atomicAdd(&sw.done[a], 1);
    s_last = prev == (int)gridDim.y - 1;
    if (s_last) sw.done[a] = 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  node_tail(pr, sw, a, t);
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
    sw.done[a] = 0;
  }
}

// Bests after evaluation t (Algorithm 1, strict "<", particles in increasing
// order), then -- if t < T -- the synchronous move to iteration t+1.
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

static size_t hist_smem_bytes(const Problem& pr) {
  const size_t hist = (hist_particle_bytes(pr.crit, pr.B, pr.K) * kWP + 127) & ~(size_t)127;
  return hist + 2 * stage_bytes(pr.w != nullptr);
}

cudaError_t prepare_eval_kernels(const Problem& pr) {
  cudaError_t e = cudaFuncSetAttribute(k_project,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kProjSmem);
  if (e) return e;
  if ((e = cudaFuncSetAttribute(k_hist_scan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)hist_smem_bytes(pr))))
    return e;
  return cudaFuncSetAttribute(k_hist_scan, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

cudaError_t launch_swarm_init(const Problem& pr, const Swarm& sw,
                              const NodeDesc* nodes, int A, SwarmCoef co,
                              cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  k_swarm_init<<<A, kThreads, 0, st>>>(pr, sw, nodes, co);
  return cudaGetLastError();
}

cudaError_t launch_project(const Problem& pr, const Swarm& sw, const WorkTile* tiles,
                           int n_tiles, int grid_cap, cudaStream_t st) {
  const int n_units = n_tiles * pr.G;
  if (n_units <= 0) return cudaSuccess;
  const int grid = n_units < grid_cap ? n_units : grid_cap;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = kProjSmem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_project, pr, sw, tiles, n_units);
}

int hist_split(const Problem& pr, int A, int64_t max_len, int n_sm, int max_cluster) {
  // clusters of S CTAs per (node, particle group): enough CTAs to fill the
  // GPU twice, slices of at least 1024 entries
  const int groups = (pr.P + kWP - 1) / kWP;
  int S = 1;
  while (2 * S <= max_cluster && (int64_t)A * groups * S < 2LL * n_sm &&
         max_len / (2 * S) >= 1024)
    S *= 2;
  return S;
}

int hist_max_cluster(const Problem& pr) {
  // largest power-of-two cluster (<= 16) the device can schedule for this kernel
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = hist_smem_bytes(pr);
  int n = 0;
  if (cudaOccupancyMaxPotentialClusterSize(&n, k_hist_scan, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 8;
  }
  int S = 1;
  while (2 * S <= n && 2 * S <= 16) S *= 2;
  return S;
}

cudaError_t launch_hist_scan(const Problem& pr, const Swarm& sw, const NodeDesc* nodes,
                             int A, int S, int32_t* bins_out, int t, SwarmCoef co,
                             int do_update, cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(A * S), (unsigned)((pr.P + kWP - 1) / kWP), 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = hist_smem_bytes(pr);
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
  return cudaLaunchKernelEx(&cfg, k_hist_scan, pr, sw, nodes, bins_out, t, co, do_update);
}

cudaError_t launch_move(const Problem& pr, const Swarm& sw, const NodeDesc* nodes, int A,
                        int t, SwarmCoef co, cudaStream_t st) {
  const int64_t items = (int64_t)A * pr.P * ((pr.d + 3) / 4);
  if (items <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((items + 127) / 128), 1, 1);
  cfg.blockDim = dim3(128, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_move, pr, sw, nodes, A, t, co);
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
