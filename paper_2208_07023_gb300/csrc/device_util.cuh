// Device helpers shared by the kernels of libslm: programmatic dependent
// launch, ordered-int floats, score comparison, bulk copies with bounded
// mbarrier waits, and the pbest step of Algorithm 1.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

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


// c ln c of a count, 0 ln 0 = 0 (natural logarithm, double precision).
__device__ __forceinline__ double xlogx(uint32_t c) {
  const double x = (double)c;
  return c ? x * log(x) : 0.0;
}

// bin(z) = min(B - 1, floor((z - zmin) * inv_w)), clamped at 0; FP32 with one
// rounding per operation (no contraction into a fused multiply-add).
__device__ __forceinline__ int bin_of(float z, float zmin, float inv_w, int B) {
  const float off = __fsub_rn(z, zmin);
  const float pos = __fmul_rn(off, inv_w);
  int b = (int)floorf(pos);
  b = b > B - 1 ? B - 1 : b;
  return b < 0 ? 0 : b;
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
// 2D tiled tensor copy global -> this CTA's shared memory: the box of the
// tensor map `tmap` (address of a __grid_constant__ kernel parameter) at
// element coordinates (x innermost, y); out-of-range elements read as zero.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_addr(bar))
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


// ---- per-thread async copies ---------------------------------------------------

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

// Row of entry e (e < pr.E): gathered from the base rows when pr.gidx is set.
__device__ __forceinline__ const float* row_of(const Problem& pr, int64_t e) {
  return pr.gidx ? pr.Xg + (int64_t)__ldg(pr.gidx + e) * pr.d : pr.X + e * pr.d;
}



// Score written by another CTA of this grid: read through L2.
__device__ __forceinline__ EvalRes ldcg_res(const EvalRes* r) {
  EvalRes o;
  const unsigned long long* w = reinterpret_cast<const unsigned long long*>(r);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(&o);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(EvalRes) / 8); ++i) d[i] = __ldcg(w + i);
  return o;
}

// Algorithm 1, gbest step of node a after evaluation t, as seen by one warp:
// the particle with the best score strictly better than gold (at t = 0 every
// particle, gold unset), ties to the lower index; -1 if none. Lane 0 also
// returns that particle's score in *best_res. With l2, the scores are read
// through L2 (written by other CTAs of the grid).
//
// The reduction runs on the double loss, which every score carries and which
// is a rounding of the exact loss (Gini: of 1 - Q / n), so it orders scores
// like the exact comparison except, possibly, among losses within a few
// units in the last place of each other. The candidates within 8 ulps of the
// smallest loss are then compared exactly (better(), index ties), which gives
// the result of an exact argmin over all candidates.
__device__ __forceinline__ uint64_t loss_key(const EvalRes& e) {
  // losses are >= 0: their bit patterns order like their values; invalid
  // scores last
  return e.valid ? (uint64_t)__double_as_longlong(e.loss) : ~0ull;
}

// The warp's choice among its lanes' candidates: lane l proposes particle bi
// (-1: none) with score be; returns the chosen particle (-1 when no lane has
// a candidate) and, in lane 0, its score into *best_res (be of lane 0 when
// there is none).
__device__ int gbest_select(const Problem& pr, int bi, const EvalRes& be, EvalRes* best_res) {
  const int lane = threadIdx.x & 31;
  const unsigned cand = __ballot_sync(0xffffffffu, bi >= 0);
  if (!cand) {  // nobody beat gold
    if (lane == 0) *best_res = be;
    return -1;
  }
  // smallest double loss over the lanes' candidates
  const uint64_t key = bi >= 0 ? loss_key(be) : ~0ull;
  uint64_t kmin = key;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t o = __shfl_xor_sync(0xffffffffu, kmin, off);
    kmin = o < kmin ? o : kmin;
  }
  // the candidates near the smallest loss (all of them when no candidate is
  // valid), compared exactly in lane order
  const bool near = bi >= 0 && (kmin == ~0ull || key <= kmin + 8);
  unsigned m = __ballot_sync(0xffffffffu, near);
  int wi = __ffs(m) - 1;
  int wb = __shfl_sync(0xffffffffu, bi, wi);
  m &= m - 1;
  while (m) {  // rare: several candidates within a few ulps
    const int li = __ffs(m) - 1;
    m &= m - 1;
    const int ob = __shfl_sync(0xffffffffu, bi, li);
    const EvalRes o = shfl_res(be, li);
    const EvalRes w = shfl_res(be, wi);
    if (better(o, w, pr.crit) || (!better(w, o, pr.crit) && ob < wb)) {
      wi = li;
      wb = ob;
    }
  }
  const EvalRes w = shfl_res(be, wi);
  if (lane == 0) *best_res = w;
  return wb;
}

// Lane l's candidate among particles l and l + 32 (scores e0, e1; in that
// order), against the gbest score gold of the previous step (every valid
// score is a candidate at t = 0).
__device__ __forceinline__ void gbest_consider(const Problem& pr, const EvalRes& gold, int t,
                                               int p, const EvalRes& e, int* bi, EvalRes* be) {
  if (!(t == 0 || better(e, gold, pr.crit))) return;
  if (*bi < 0 || better(e, *be, pr.crit)) {
    *bi = p;
    *be = e;
  }
}

__device__ int gbest_argmin(const Problem& pr, const EvalRes* cur, const EvalRes& gold, int t,
                            EvalRes* best_res, bool l2 = false) {
  const int lane = threadIdx.x & 31;
  int bi = -1;
  EvalRes be = invalid_res();
  // two records per lane in flight, considered in particle order
  for (int p = lane; p < pr.P; p += 64) {
    const bool two = p + 32 < pr.P;
    const EvalRes e0 = l2 ? ldcg_res(cur + p) : cur[p];
    EvalRes e1 = e0;
    if (two) e1 = l2 ? ldcg_res(cur + p + 32) : cur[p + 32];
    gbest_consider(pr, gold, t, p, e0, &bi, &be);
    if (two) gbest_consider(pr, gold, t, p + 32, e1, &bi, &be);
  }
  return gbest_select(pr, bi, be, best_res);
}

// Folded searches (Swarm::imp): records that score `res` of a particle of
// node a in evaluation t beats the gbest score held after evaluation t - 1
// (every valid score does at t = 0), the gbest step's rule (Algorithm 1).
__device__ __forceinline__ void mark_improvement(const Problem& pr, const Swarm& sw, int a, int t,
                                                 const EvalRes& res) {
  if (!sw.imp || !res.valid) return;
  const bool beats =
      t == 0 || better(res, ldcg_res(sw.gb + (int64_t)((t + 1) & 1) * sw.n_nodes + a), pr.crit);
  if (beats) atomicOr(sw.imp + (int64_t)(t & 1) * sw.n_nodes + a, 1);
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


__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Four consecutive features j0..j0+3 (j0 % 4 == 0) of particle p of node a as
// bfloat16 MMA operands: posb[a, Pp * dp] in the K-major core-matrix layout
// (16-feature steps of Pp x 16, 8-row groups of 128 elements, two 8-feature
// halves of 64, rows of 8).
__device__ __forceinline__ void store_posb4(uint16_t* posb, int Pp, int dp, int a, int p, int j0,
                                            const float (&v)[4]) {
  const int64_t off = (int64_t)a * Pp * dp + (int64_t)(j0 >> 4) * Pp * 16 + (p >> 3) * 128 +
                      ((j0 >> 3) & 1) * 64 + (p & 7) * 8 + (j0 & 7);
  uint2 u;
  u.x = pack_bf16x2(v[0], v[1]);
  u.y = pack_bf16x2(v[2], v[3]);
  *reinterpret_cast<uint2*>(posb + off) = u;
}

}  // namespace
}  // namespace slm
