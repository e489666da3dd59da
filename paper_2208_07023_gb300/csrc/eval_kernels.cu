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
//    A persistent grid walks (tile of kTS = 256 rows, group of PG = 8..48
//    particles, picked per problem shape by the autotuner) work units; rows and positions stream through shared memory
//    in kKC = 32-feature chunks with double-buffered cp.async copies. Each
//    thread owns a 4 x 4 register tile (rows w*32 + sg + 8i, particles
//    pg + 4j) and accumulates over the features in increasing order, so every
//    z is the same sequence of fused multiply-adds whatever the tiling. The
//    per-(node, particle) range is folded in with ordered-int atomics and z is
//    written to an L2-resident buffer.
//  * k_hist_scan: one CTA per (node, particle) bins the node's z into
//    warp-private shared histograms, merges them and scans the edges.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <float.h>
#include <limits.h>
#include <math.h>

#include <cooperative_groups.h>

#include <mutex>
#include <vector>

#include "philox.cuh"
#include "slm_internal.cuh"
#include "device_util.cuh"
#include "scan_util.cuh"

namespace slm {

namespace {


// Polls of the histogram kernel's first wait on each staged piece (the
// drain of copies in flight after a failed wait keeps kWaitPolls). Lowered
// only to test the timeout path: at 0 every piece's wait gives up at once,
// the kernel drains its copies, records the error word and ends normally.
__device__ int d_first_wait_polls = kWaitPolls;

// c ln c for c < kXlogxTab from a table the device builds once with xlogx
// itself (identical values): the entropy scans then read L2 instead of
// evaluating double-precision logarithms, which are scarce on this GPU.
__device__ const double* d_xlogx_tab = nullptr;

__global__ void k_xlogx_table(double* tab, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) tab[i] = xlogx((uint32_t)i);
}

__device__ __forceinline__ double xlogx_t(uint32_t c) {
  const double* t = d_xlogx_tab;
  return (t && c < (uint32_t)kXlogxTab) ? __ldg(t + c) : xlogx(c);
}


// ---- threshold scans (one warp, one particle) ----------------------------------

// Classification threshold scan of one particle by the whole CTA.
// h: [B][K] counts in shared memory (turned into per-class prefix sums in
// place). Edge b splits bins < b from bins >= b; an edge whose bin b-1 is
// empty repeats edge b-1's partition and is skipped (the lower edge wins).
template <int CRIT>
__device__ EvalRes block_scan_cls(uint32_t* h, int B, int K, int min_leaf, ScanScratch& sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // 1. per-class inclusive prefix over bins: warp w takes classes w, w+8, ...;
  //    lane l owns bins [l*bpl, (l+1)*bpl)
  const int bpl = (B + 31) >> 5;
  for (int k = warp; k < K; k += kThreads / 32) {
    uint32_t v[kMaxBins / 32];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kMaxBins / 32; ++i) {
      const int j = lane * bpl + i;
      v[i] = (i < bpl && j < B) ? h[j * K + k] : 0u;
      sum += v[i];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += u;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int i = 0; i < kMaxBins / 32; ++i) {
      const int j = lane * bpl + i;
      run += v[i];
      if (i < bpl && j < B) h[j * K + k] = run;
    }
  }
  __syncthreads();
  // 2. one thread per edge b = 1 + tid
  const uint32_t* tot = h + (B - 1) * K;
  uint32_t ntot = 0;
  for (int k = 0; k < K; ++k) ntot += tot[k];
  const int b = 1 + threadIdx.x;
  uint32_t nl = 0;
  uint64_t sl = 0, sr = 0;
  double hl = 0.0, hr = 0.0;
  if (b < B) {
    const uint32_t* row = h + (b - 1) * K;
    for (int k = 0; k < K; ++k) {
      const uint32_t l = row[k], r = tot[k] - l;
      nl += l;
      if (CRIT == SLM_GINI) {
        sl += (uint64_t)l * l;
        sr += (uint64_t)r * r;
      } else {
        hl += xlogx_t(l);
        hr += xlogx_t(r);
      }
    }
    sc.nl[threadIdx.x] = nl;
  }
  __syncthreads();
  const uint32_t prev = (b >= 2 && b < B) ? sc.nl[threadIdx.x - 1] : 0u;
  const uint32_t nr = ntot - nl;
  uint64_t bn = 0, bd = 0;
  double bl = 0.0;
  int bb = -1;
  if (b < B && nl != prev && nl >= (uint32_t)min_leaf && nr >= (uint32_t)min_leaf) {
    bb = b;
    if (CRIT == SLM_GINI) {
      bn = sl * nr + sr * nl;
      bd = (uint64_t)nl * nr;
    } else {
      // compared after the division by n, as the criterion is defined
      bl = ((xlogx_t(nl) - hl) + (xlogx_t(nr) - hr)) / (double)ntot;
    }
  }
  block_argmin<CRIT>(bn, bd, bl, bb, sc);
  if (threadIdx.x == 0) {
    EvalRes res = invalid_res();
    const int wb = sc.wb[0];
    if (wb >= 0) {
      res.valid = 1;
      res.bin = wb;
      res.nl = sc.nl[wb - 1];
      res.nr = ntot - sc.nl[wb - 1];
      if (CRIT == SLM_GINI) {
        res.num = sc.wn[0];
        res.den = sc.wd[0];
        const uint64_t nden = (uint64_t)ntot * res.den;
        res.loss = (double)(nden - res.num) / (double)nden;
      } else {
        res.loss = sc.wl[0];
      }
    }
    sc.res = res;
  }
  __syncthreads();
  return sc.res;
}


// ---- projection -------------------------------------------------------------------

constexpr size_t kProjSmem = sizeof(float) * 2 * (kTS * kXS + kPGMax * kXS);


// Stages one kKC-feature chunk of a work unit's rows and PG positions.
template <int PG>
__device__ __forceinline__ void stage_chunk(const Problem& pr, const Swarm& sw,
                                            const WorkTile& wt, int g, int k0,
                                            bool vec, float* xb, float* ab) {
  const int d = pr.d;
  const int kc = min(kKC, d - k0);
  const float* pos = sw.pos + ((int64_t)wt.node * pr.Pp + g * PG) * d;
  if (vec) {
    for (int q = threadIdx.x; q < kTS * (kKC / 4); q += kThreads) {
      const int r = q >> 3, cc = (q & 7) * 4;
      const bool ok = r < wt.rows && cc < kc;
      const float* src = ok ? row_of(pr, wt.row0 + r) + k0 + cc : pr.X;
      cp_async16(xb + r * kXS + cc, src, ok ? 16 : 0);
    }
    for (int q = threadIdx.x; q < PG * (kKC / 4); q += kThreads) {
      const int p = q >> 3, cc = (q & 7) * 4;
      const bool ok = cc < kc && g * PG + p < pr.Pp;
      cp_async16(ab + p * kXS + cc, ok ? pos + (int64_t)p * d + k0 + cc : pos, ok ? 16 : 0);
    }
  } else {
    for (int q = threadIdx.x; q < kTS * kKC; q += kThreads) {
      const int r = q >> 5, cc = q & 31;
      const bool ok = r < wt.rows && cc < kc;
      const float* src = ok ? row_of(pr, wt.row0 + r) + k0 + cc : pr.X;
      cp_async4(xb + r * kXS + cc, src, ok ? 4 : 0);
    }
    for (int q = threadIdx.x; q < PG * kKC; q += kThreads) {
      const int p = q >> 5, cc = q & 31;
      const bool ok = cc < kc && g * PG + p < pr.Pp;
      cp_async4(ab + p * kXS + cc, ok ? pos + (int64_t)p * d + k0 + cc : pos, ok ? 4 : 0);
    }
  }
  cp_async_commit();
}

// PG particles per work unit (8, 16, 24, 32 or 48; G = Pp / PG groups): each
// thread owns 4 rows x PG/4 particles. Wider groups read a tile's rows once
// for more particles (fewer passes over rows that do not stay in L2);
// narrower ones give more units to spread over the SMs.
template <int PG>
__global__ void __launch_bounds__(kThreads, 2)
    k_project(Problem pr, Swarm sw, const WorkTile* __restrict__ tiles, int n_units) {
  constexpr int PJ = PG / 4;
  static_assert(PG % 8 == 0 && PG <= kPGMax, "particle group");
  extern __shared__ __align__(16) float smf[];
  float* xs0 = smf;
  float* xs1 = smf + kTS * kXS;
  float* as0 = smf + 2 * kTS * kXS;
  float* as1 = as0 + kPGMax * kXS;
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
    stage_chunk<PG>(pr, sw, tiles[u / G], u % G, 0, vec, xs0, as0);
  }
  float acc[4][PJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < PJ; ++j) acc[i][j] = 0.0f;

  for (int s = 0; s < n_st; ++s) {
    const int ui = s / nk, c = s - ui * nk;
    const int u = blockIdx.x + ui * gridDim.x;
    if (s + 1 < n_st) {
      const int ui1 = (s + 1) / nk, c1 = (s + 1) - ui1 * nk;
      const int u1 = blockIdx.x + ui1 * gridDim.x;
      stage_chunk<PG>(pr, sw, tiles[u1 / G], u1 % G, c1 * kKC, vec, (s & 1) ? xs0 : xs1,
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
    if constexpr (PJ <= 4) {
#pragma unroll 2
      for (int k = 0; k < kc4; k += 4) {
        float4 xv[4], av[PJ];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          xv[i] = *reinterpret_cast<const float4*>(xr + i * 8 * kXS + k);
#pragma unroll
        for (int j = 0; j < PJ; ++j)
          av[j] = *reinterpret_cast<const float4*>(ar + j * 4 * kXS + k);
        // feature-outer: every accumulator takes features k..k+3 in order,
        // and consecutive FMAs go to independent accumulators
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < PJ; ++j) acc[i][j] = fmaf(xv[i].x, av[j].x, acc[i][j]);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < PJ; ++j) acc[i][j] = fmaf(xv[i].y, av[j].y, acc[i][j]);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < PJ; ++j) acc[i][j] = fmaf(xv[i].z, av[j].z, acc[i][j]);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < PJ; ++j) acc[i][j] = fmaf(xv[i].w, av[j].w, acc[i][j]);
      }
    } else {
      // wide groups: two particles' 4 features at a time keep the live
      // registers at the accumulators plus the rows and two position vectors
      for (int k = 0; k < kc4; k += 4) {
        float4 xv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          xv[i] = *reinterpret_cast<const float4*>(xr + i * 8 * kXS + k);
#pragma unroll
        for (int j = 0; j < PJ; j += 2) {
          const float4 a0 = *reinterpret_cast<const float4*>(ar + j * 4 * kXS + k);
          const float4 a1 = *reinterpret_cast<const float4*>(ar + (j + 1) * 4 * kXS + k);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[i][j] = fmaf(xv[i].x, a0.x, acc[i][j]);
            acc[i][j + 1] = fmaf(xv[i].x, a1.x, acc[i][j + 1]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[i][j] = fmaf(xv[i].y, a0.y, acc[i][j]);
            acc[i][j + 1] = fmaf(xv[i].y, a1.y, acc[i][j + 1]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[i][j] = fmaf(xv[i].z, a0.z, acc[i][j]);
            acc[i][j + 1] = fmaf(xv[i].z, a1.z, acc[i][j + 1]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[i][j] = fmaf(xv[i].w, a0.w, acc[i][j]);
            acc[i][j + 1] = fmaf(xv[i].w, a1.w, acc[i][j + 1]);
          }
        }
      }
    }
    if (c == nk - 1) {
      // tile complete: fold the range, store z
      const WorkTile wt = tiles[u / G];
      const int g = u % G;
#pragma unroll
      for (int j = 0; j < PJ; ++j) {
        const int p = g * PG + pg + 4 * j;
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
        for (int j = 0; j < PJ; ++j) acc[i][j] = 0.0f;
    }
    __syncthreads();  // buffer s&1 is refilled by the next stage's copies
  }
}

// ---- projection with tensor-map tile copies (TMA) ----------------------------------
//
// The same work units, arithmetic and epilogue as k_project, for rows that
// are contiguous in pr.X (no gather) with d % 4 == 0: thread 0 fetches each
// kKC-feature chunk of a unit as two 2D boxes of tensor maps (kTS rows x 32
// features of X, PG positions x 32 features) into a two-stage ring, the
// copies completing on an mbarrier; 128-byte swizzle (16-byte chunk c of
// smem row r stored at c ^ (r mod 8)) keeps the float4 reads of 8 lanes on
// 8 consecutive rows on distinct banks. Features past d and rows past the
// tensor's end arrive as zeros. Every wait is bounded; a copy that does not
// land sets the error word (kErrCopyTimeout) and ends the kernel after the copies in flight.

constexpr int kTmaRowBytes = kKC * 4;                   // one box row: 128 B
constexpr int kTmaXBytes = kTS * kTmaRowBytes;          // 32 KB
constexpr int kTmaABytes = kPGMax * kTmaRowBytes;       // 6 KB (room for PG <= 48)
constexpr size_t kProjTmaSmem = 2 * (kTmaXBytes + kTmaABytes) + 1024;  // + alignment

template <int PG>
__global__ void __launch_bounds__(kThreads, 2)
    k_project_tma(const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap ta,
                  Problem pr, Swarm sw, const WorkTile* __restrict__ tiles, int n_units) {
  constexpr int PJ = PG / 4;
  static_assert(PG % 8 == 0 && PG <= kPGMax, "particle group");
  extern __shared__ unsigned char tsm_raw[];
  __shared__ __align__(8) uint64_t s_bar[2];
  // the swizzle pattern repeats every 1024 bytes: stage buffers start on it
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tsm_raw) + 1023) & ~uintptr_t(1023));
  // stage b: rows at base + b * kTmaXBytes, positions after both row stages
  auto xstage = [&](int b) { return reinterpret_cast<float*>(base + b * kTmaXBytes); };
  auto astage = [&](int b) {
    return reinterpret_cast<float*>(base + 2 * kTmaXBytes + b * kTmaABytes);
  };
  pdl_trigger();
  pdl_wait();
  if ((int)blockIdx.x >= n_units) return;
  const int d = pr.d, G = pr.G;
  const int nk = (d + kKC - 1) / kKC;
  const int my_units = (n_units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;
  const int n_st = my_units * nk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sg = lane & 7, pg = lane >> 3;
  const uint32_t stage_bytes = (uint32_t)(kTmaXBytes + PG * kTmaRowBytes);
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int s) {
    const int ui = s / nk, c = s - ui * nk;
    const int u = blockIdx.x + ui * gridDim.x;
    const WorkTile wt = tiles[u / G];
    const int g = u % G;
    uint64_t* bar = &s_bar[s & 1];
    fence_proxy_async();
    mbar_expect_tx(bar, stage_bytes);
    tma_load_2d(xstage(s & 1), &tx, c * kKC, (int)wt.row0, bar);
    tma_load_2d(astage(s & 1), &ta, c * kKC, wt.node * pr.Pp + g * PG, bar);
  };
  if (threadIdx.x == 0) issue(0);
  float acc[4][PJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < PJ; ++j) acc[i][j] = 0.0f;

  for (int s = 0; s < n_st; ++s) {
    const int ui = s / nk, c = s - ui * nk;
    const int u = blockIdx.x + ui * gridDim.x;
    // the other stage was released by the barrier that ended step s - 1
    if (threadIdx.x == 0 && s + 1 < n_st) issue(s + 1);
    const bool ok = mbar_wait(&s_bar[s & 1], (uint32_t)((s >> 1) & 1), kWaitPolls);
    if (__syncthreads_or(!ok)) {
      // a copy did not land: record it, give the copies in flight a bounded
      // chance to finish, and end
      if (threadIdx.x == 0) {
        if (sw.err) atomicExch(sw.err, kErrCopyTimeout);
        if (s + 1 < n_st) mbar_wait(&s_bar[(s + 1) & 1], (uint32_t)(((s + 1) >> 1) & 1),
                                    kWaitPolls);
      }
      return;
    }
    const float* xb = xstage(s & 1);
    const float* ab = astage(s & 1);
    const int kc4 = (min(kKC, d - c * kKC) + 3) & ~3;
    // rows warp*32 + sg + 8i all have r mod 8 = sg; particle pg + 4j has
    // (pg + 4j) mod 8 = pg + 4 (j & 1)
    const float* xr = xb + (warp * 32 + sg) * kKC;
    const float* ar = ab + pg * kKC;
    if constexpr (PJ <= 4) {
#pragma unroll 2
      for (int k = 0; k < kc4; k += 4) {
        const int ch = k >> 2;
        float4 xv[4], av[PJ];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          xv[i] = *reinterpret_cast<const float4*>(xr + i * 8 * kKC + ((ch ^ sg) << 2));
#pragma unroll
        for (int j = 0; j < PJ; ++j)
          av[j] = *reinterpret_cast<const float4*>(ar + j * 4 * kKC +
                                                   ((ch ^ (pg + 4 * (j & 1))) << 2));
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < PJ; ++j) acc[i][j] = fmaf(xv[i].x, av[j].x, acc[i][j]);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < PJ; ++j) acc[i][j] = fmaf(xv[i].y, av[j].y, acc[i][j]);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < PJ; ++j) acc[i][j] = fmaf(xv[i].z, av[j].z, acc[i][j]);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < PJ; ++j) acc[i][j] = fmaf(xv[i].w, av[j].w, acc[i][j]);
      }
    } else {
      for (int k = 0; k < kc4; k += 4) {
        const int ch = k >> 2;
        float4 xv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          xv[i] = *reinterpret_cast<const float4*>(xr + i * 8 * kKC + ((ch ^ sg) << 2));
#pragma unroll
        for (int j = 0; j < PJ; j += 2) {
          const float4 a0 =
              *reinterpret_cast<const float4*>(ar + j * 4 * kKC + ((ch ^ pg) << 2));
          const float4 a1 = *reinterpret_cast<const float4*>(ar + (j + 1) * 4 * kKC +
                                                             ((ch ^ (pg + 4)) << 2));
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[i][j] = fmaf(xv[i].x, a0.x, acc[i][j]);
            acc[i][j + 1] = fmaf(xv[i].x, a1.x, acc[i][j + 1]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[i][j] = fmaf(xv[i].y, a0.y, acc[i][j]);
            acc[i][j + 1] = fmaf(xv[i].y, a1.y, acc[i][j + 1]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[i][j] = fmaf(xv[i].z, a0.z, acc[i][j]);
            acc[i][j + 1] = fmaf(xv[i].z, a1.z, acc[i][j + 1]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[i][j] = fmaf(xv[i].w, a0.w, acc[i][j]);
            acc[i][j + 1] = fmaf(xv[i].w, a1.w, acc[i][j + 1]);
          }
        }
      }
    }
    if (c == nk - 1) {
      // tile complete: fold the range, store z (k_project's epilogue)
      const WorkTile wt = tiles[u / G];
      const int g = u % G;
#pragma unroll
      for (int j = 0; j < PJ; ++j) {
        const int p = g * PG + pg + 4 * j;
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
        for (int j = 0; j < PJ; ++j) acc[i][j] = 0.0f;
    }
    __syncthreads();  // stage s & 1 is refilled by the copies issued at step s + 1
  }
}

// ---- swarm update ----------------------------------------------------------------



// The particle with the worst score of node a (invalid scores worst, ties
// to the lower index), as seen by one warp; every lane returns it.
__device__ int worst_argmax(const Problem& pr, const EvalRes* cur) {
  const int lane = threadIdx.x & 31;
  int wi = -1;
  EvalRes we = invalid_res();
  for (int p = lane; p < pr.P; p += 32) {
    const EvalRes e = cur[p];
    if (wi < 0 || better(we, e, pr.crit)) {
      wi = p;
      we = e;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const int oi = __shfl_xor_sync(0xffffffffu, wi, off);
    const EvalRes o = shfl_res(we, lane ^ off);
    bool take;
    if (oi < 0)
      take = false;
    else if (wi < 0)
      take = true;
    else if (better(we, o, pr.crit))
      take = true;
    else if (better(o, we, pr.crit))
      take = false;
    else
      take = oi < wi;
    if (take) {
      wi = oi;
      we = o;
    }
  }
  return wi;
}

// Eq. pso-1 for features 4q..4q+3 of particle pi of node a, to iteration t+1:
// v <- omega v + (c1 r1)(pB - x) + (c2 r2)(gB - x);  x <- x + v. pbp: the
// node's pbest rows, gsrc: gB. With sw.posb the new positions are also
// written as bfloat16 MMA operands.
__device__ __forceinline__ void move_item(const Problem& pr, const Swarm& sw, const SwarmCoef& co,
                                          uint32_t uid, int a, int t, int pi, int q,
                                          const float* pbp, const float* gsrc) {
  const int d = pr.d, Pp = pr.Pp;
  const uint32_t k0 = (uint32_t)co.seed, k1 = (uint32_t)(co.seed >> 32);
  const U4 r1 = philox4x32_10(uid, (uint32_t)(t + 1), (uint32_t)pi,
                              (uint32_t)q | (kR1 << 24), k0, k1);
  const U4 r2 = philox4x32_10(uid, (uint32_t)(t + 1), (uint32_t)pi,
                              (uint32_t)q | (kR2 << 24), k0, k1);
  const int64_t row = (int64_t)pi * d;
  float* pos = sw.pos + (int64_t)a * Pp * d + row;
  float* vel = sw.vel + (int64_t)a * Pp * d + row;
  float xn[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = 4 * q + c;
    if (j >= d) break;
    const float x = pos[j], v = vel[j];
    const float inertia = __fmul_rn(co.inertia, v);
    const float cog =
        __fmul_rn(__fmul_rn(co.c1, uniform24(r1.v[c])), __fsub_rn(pbp[row + j], x));
    const float soc = __fmul_rn(__fmul_rn(co.c2, uniform24(r2.v[c])), __fsub_rn(gsrc[j], x));
    const float vn = __fadd_rn(__fadd_rn(inertia, cog), soc);
    vel[j] = vn;
    xn[c] = __fadd_rn(x, vn);
    pos[j] = xn[c];
  }
  if (sw.posb) store_posb4(sw.posb, Pp, pr.dp, a, pi, 4 * q, xn);
}

// The terms of Eq. pso-1 for particle pi of node a that do not depend on gB,
// after the pbest step of evaluation t (one warp; t < T): for every feature j,
// ic = omega v + (c1 r1)(pB - x) and s2 = c2 r2, r1 and r2 the draws of the
// move to t + 1 (counter (uid, t + 1, pi, j/4)), each operation rounded as in
// move_item; k_step finishes the move with v' = ic + s2 (gB - x), x' = x + v'.
__device__ __forceinline__ void premove_particle(const Problem& pr, const Swarm& sw, uint32_t uid,
                                                 int a, int t, int pi) {
  const int lane = threadIdx.x & 31;
  const int d = pr.d, d4 = (d + 3) >> 2;
  const SwarmCoef& co = sw.co;
  const uint32_t k0 = (uint32_t)co.seed, k1 = (uint32_t)(co.seed >> 32);
  const int64_t row = ((int64_t)a * pr.Pp + pi) * d;
  const float* x = sw.pos + row;
  const float* v = sw.vel + row;
  const float* pb = sw.pbest + row;
  for (int q = lane; q < d4; q += 32) {
    const U4 r1 = philox4x32_10(uid, (uint32_t)(t + 1), (uint32_t)pi,
                                (uint32_t)q | (kR1 << 24), k0, k1);
    const U4 r2 = philox4x32_10(uid, (uint32_t)(t + 1), (uint32_t)pi,
                                (uint32_t)q | (kR2 << 24), k0, k1);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = 4 * q + c;
      if (j >= d) break;
      const float xj = x[j];
      const float inertia = __fmul_rn(co.inertia, v[j]);
      const float cog = __fmul_rn(__fmul_rn(co.c1, uniform24(r1.v[c])), __fsub_rn(pb[j], xj));
      sw.ic[row + j] = __fadd_rn(inertia, cog);
      sw.s2[row + j] = __fmul_rn(co.c2, uniform24(r2.v[c]));
    }
  }
}

// Fuzzy memberships of the evolutionary factor f in the adaptive PSO states
// (1 exploration, 2 exploitation, 3 convergence, 4 jumping out).
__device__ float apso_mu(int state, float f) {
  switch (state) {
    case 1:
      if (f <= 0.4f) return 0.0f;
      if (f <= 0.6f) return __fsub_rn(__fmul_rn(5.0f, f), 2.0f);
      if (f <= 0.7f) return 1.0f;
      if (f <= 0.8f) return __fadd_rn(__fmul_rn(-10.0f, f), 8.0f);
      return 0.0f;
    case 2:
      if (f <= 0.2f) return 0.0f;
      if (f <= 0.3f) return __fsub_rn(__fmul_rn(10.0f, f), 2.0f);
      if (f <= 0.4f) return 1.0f;
      if (f <= 0.6f) return __fadd_rn(__fmul_rn(-5.0f, f), 3.0f);
      return 0.0f;
    case 3:
      if (f <= 0.1f) return 1.0f;
      if (f <= 0.3f) return __fadd_rn(__fmul_rn(-5.0f, f), 1.5f);
      return 0.0f;
    default:
      if (f <= 0.7f) return 0.0f;
      if (f <= 0.9f) return __fsub_rn(__fmul_rn(5.0f, f), 3.5f);
      return 1.0f;
  }
}

// Adaptive PSO (Sec. III-B; the published rules of the cited APSO method),
// one CTA per node after evaluation t, in place of k_move:
// 1. the gbest step (k_move's rule), then the elite candidate scored in this
//    evaluation (slot P): gB and the gB particle's personal best if strictly
//    better, else the worst particle's position (and personal best if beaten);
// for t < T:
// 2. each particle's mean distance d_i to the others (every squared distance
//    a sequential fused multiply-add sum over the features, then the square
//    roots added in increasing j, all in float with one rounding per
//    operation); f = (d_g - d_min) / (d_max - d_min); the state from f's
//    memberships (overlaps: keep the previous state, else the next in the
//    ring 1 -> 2 -> 3 -> 4 -> 1, else the larger membership, ties to the
//    lower state); the learning factors moved by delta = 0.05 + 0.05 u (u
//    the swarm draw of purpose 7 at (uid, t, 0, 0)), clamped to [1.5, 2.5]
//    and scaled to a sum of 4 when above; the inertia 1 / (1 + 1.5
//    exp(-2.6 f)) in double, rounded to float;
// 3. in the convergence state the next elite candidate (elitist learning);
// 4. the move of Eq. pso-1 with these factors.
//
// Layout: positions feature-major in shared memory (row k holds feature k of
// the Pq = P rounded up to 4 particles, 16-byte aligned), so a thread's 4 x 4
// tile of (i, j) pairs reads two float4 per feature and the lanes of a warp
// (consecutive j blocks) read consecutive 16-byte words. The rows i are taken
// in chunks of apso_rows(P, d) whose square roots go to a buffer of stride
// Pq + 1, from which thread r adds row r without bank conflicts.
__host__ __device__ inline int apso_pq(int P) { return (P + 3) & ~3; }

__host__ __device__ inline size_t apso_smem(int P, int d, int R) {
  const int Pq = apso_pq(P);
  return sizeof(float) * ((size_t)d * Pq + (size_t)R * (Pq + 1));
}

// Rows per chunk: the largest of 64, 32, 16, 8, 4 (not above Pq) whose
// buffers fit in 227 KB; 0 if none does.
inline int apso_rows(int P, int d) {
  const int Pq = apso_pq(P);
  for (int R = 64; R >= 4; R >>= 1)
    if (R <= Pq && apso_smem(P, d, R) <= 227 * 1024) return R;
  return apso_smem(P, d, 4) <= 227 * 1024 ? 4 : 0;
}

__global__ void __launch_bounds__(256)
    k_apso(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes, int t, SwarmCoef co,
           const int32_t* __restrict__ list, int A, int R) {
  extern __shared__ __align__(16) float asm_[];
  __shared__ float s_di[kMaxParticles];
  __shared__ int s_gp;
  pdl_trigger();
  pdl_wait();
  __shared__ int s_mode, s_w, s_wpb, s_k;
  __shared__ float s_g, s_c[3];
  const int a = list ? list[blockIdx.x] : (int)blockIdx.x;
  const int P = pr.P, d = pr.d, Pp = pr.Pp, Pq = apso_pq(P);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t cb = (int64_t)a * Pp;
  float* pos = sw.pos + cb * d;
  float* pbp = sw.pbest + cb * d;
  float* gbp = sw.gbest + (int64_t)a * d;
  float* erow = pos + (int64_t)P * d;  // the elite candidate's slot
  // 1. gbest step of evaluation t (the rule of k_move), then the elite
  // candidate scored in this evaluation: gB and the gB particle's personal
  // best if strictly better, else the worst particle's position (and its
  // personal best if better than it)
  if (warp == 0) {
    const EvalRes gold = sw.gb[(int64_t)((t + 1) & 1) * A + a];
    EvalRes be;
    const int bi = gbest_argmin(pr, sw.cur + cb, gold, t, &be);
    const int pending = sw.apso[a].pending;
    const int wi = pending ? worst_argmax(pr, sw.cur + cb) : -1;
    if (lane == 0) {
      EvalRes gnew = bi >= 0 ? be : gold;
      const int gp = bi >= 0 ? bi : sw.gpart[a];
      int git = bi >= 0 ? t : sw.giter[a];
      int mode = bi >= 0 ? 1 : 0, wr = -1, wpb = 0;
      if (pending) {
        const EvalRes ee = sw.cur[cb + P];
        if (better(ee, gnew, pr.crit)) {
          gnew = ee;
          git = t;
          mode = 2;
          sw.pb[cb + gp] = ee;
        } else {
          wr = wi;
          sw.cur[cb + wi] = ee;
          if (better(ee, sw.pb[cb + wi], pr.crit)) {
            sw.pb[cb + wi] = ee;
            wpb = 1;
          }
        }
        sw.apso[a].pending = 0;
      }
      sw.gb[(int64_t)(t & 1) * A + a] = gnew;
      sw.gpart[a] = gp;
      sw.giter[a] = git;
      if (sw.trace)
        sw.trace[(int64_t)a * (sw.T + 1) + t] =
            gnew.valid ? gnew.loss : __longlong_as_double(0x7ff0000000000000LL);
      s_gp = gp;
      s_mode = mode;
      s_w = wr;
      s_wpb = wpb;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    if (s_mode == 1) {
      gbp[j] = pbp[(int64_t)s_gp * d + j];
    } else if (s_mode == 2) {
      gbp[j] = erow[j];
      pbp[(int64_t)s_gp * d + j] = erow[j];
    }
    if (s_w >= 0) {
      pos[(int64_t)s_w * d + j] = erow[j];
      if (s_wpb) pbp[(int64_t)s_w * d + j] = erow[j];
    }
  }
  if (t >= sw.T) return;
  __syncthreads();
  // 2. the evolutionary state of the current positions
  float* xt = asm_;             // [d][Pq] current positions, feature-major
  float* rw = asm_ + d * Pq;    // [R][Pq + 1] square roots of a chunk of rows
  // consecutive threads take consecutive particles of one feature: the
  // shared-memory writes go to consecutive banks (the global reads are
  // strided but hit L2: the positions were written by the last move)
  for (int e = threadIdx.x; e < Pq * d; e += blockDim.x) {
    const int k = e / Pq, i = e - k * Pq;
    xt[e] = i < P ? pos[(int64_t)i * d + k] : 0.0f;
  }
  __syncthreads();
  const int nJ = Pq >> 2, ld = Pq + 1;
  for (int c0 = 0; c0 < P; c0 += R) {
    const int rows = min(R, P - c0), nI = (rows + 3) >> 2;
    for (int u = threadIdx.x; u < nI * nJ; u += blockDim.x) {
      const int ib = u / nJ, jb = u - ib * nJ;
      const int i0 = c0 + 4 * ib, j0 = 4 * jb;
      float s2[4][4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) s2[p][q] = 0.0f;
#pragma unroll 2
      for (int k = 0; k < d; ++k) {
        const float4 xi = *reinterpret_cast<const float4*>(xt + k * Pq + i0);
        const float4 xj = *reinterpret_cast<const float4*>(xt + k * Pq + j0);
        const float vi[4] = {xi.x, xi.y, xi.z, xi.w}, vj[4] = {xj.x, xj.y, xj.z, xj.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float diff = __fsub_rn(vi[p], vj[q]);
            s2[p][q] = fmaf(diff, diff, s2[p][q]);
          }
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (i0 + p < c0 + rows && j0 + q < P)
            rw[(i0 + p - c0) * ld + j0 + q] = __fsqrt_rn(s2[p][q]);
    }
    __syncthreads();
    if ((int)threadIdx.x < rows) {
      const int i = c0 + threadIdx.x;
      const float* ri = rw + threadIdx.x * ld;
      float acc = 0.0f;
      for (int j = 0; j < P; ++j)
        if (j != i) acc = __fadd_rn(acc, ri[j]);
      s_di[i] = P > 1 ? __fdiv_rn(acc, (float)(P - 1)) : 0.0f;
    }
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float dmin = s_di[0], dmax = s_di[0];
    for (int i = 1; i < P; ++i) {
      dmin = s_di[i] < dmin ? s_di[i] : dmin;
      dmax = s_di[i] > dmax ? s_di[i] : dmax;
    }
    const float dg = s_di[s_gp];
    const float f = dmax > dmin ? __fdiv_rn(__fsub_rn(dg, dmin), __fsub_rn(dmax, dmin)) : 0.0f;
    ApsoState st = sw.apso[a];
    float mu[5];
    int cand[4], nc = 0;
    for (int q = 1; q <= 4; ++q) {
      mu[q] = apso_mu(q, f);
      if (mu[q] > 0.0f) cand[nc++] = q;
    }
    int state = cand[0];
    if (nc > 1) {
      const int next = st.state % 4 + 1;
      bool has_prev = false, has_next = false;
      for (int q = 0; q < nc; ++q) {
        has_prev |= cand[q] == st.state;
        has_next |= cand[q] == next;
      }
      if (has_prev) {
        state = st.state;
      } else if (has_next) {
        state = next;
      } else {
        for (int q = 1; q < nc; ++q)
          if (mu[cand[q]] > mu[state]) state = cand[q];
      }
    }
    const uint32_t k0 = (uint32_t)co.seed, k1 = (uint32_t)(co.seed >> 32);
    const U4 r = philox4x32_10(nodes[a].uid, (uint32_t)t, 0u, kApso << 24, k0, k1);
    const float delta = __fadd_rn(0.05f, __fmul_rn(0.05f, uniform24(r.v[0])));
    const float h = __fmul_rn(0.5f, delta);
    float c1 = st.c1, c2 = st.c2;
    if (state == 1) {
      c1 = __fadd_rn(c1, delta);
      c2 = __fsub_rn(c2, delta);
    } else if (state == 2) {
      c1 = __fadd_rn(c1, h);
      c2 = __fsub_rn(c2, h);
    } else if (state == 3) {
      c1 = __fadd_rn(c1, h);
      c2 = __fadd_rn(c2, h);
    } else {
      c1 = __fsub_rn(c1, delta);
      c2 = __fadd_rn(c2, delta);
    }
    c1 = c1 < 1.5f ? 1.5f : c1 > 2.5f ? 2.5f : c1;
    c2 = c2 < 1.5f ? 1.5f : c2 > 2.5f ? 2.5f : c2;
    const float sum = __fadd_rn(c1, c2);
    if (sum > 4.0f) {
      c1 = __fdiv_rn(__fmul_rn(4.0f, c1), sum);
      c2 = __fdiv_rn(__fmul_rn(4.0f, c2), sum);
    }
    st.state = state;
    st.c1 = c1;
    st.c2 = c2;
    st.w = (float)__ddiv_rn(1.0, __dadd_rn(1.0, __dmul_rn(1.5, exp(__dmul_rn(-2.6, (double)f)))));
    st.pending = state == 3;
    sw.apso[a] = st;
    s_mode = st.pending;
    s_c[0] = st.w;
    s_c[1] = st.c1;
    s_c[2] = st.c2;
  } else if (threadIdx.x == 32) {
    // elitist learning's step, beside thread 0's state update: coordinate
    // k = floor(u1 d), g = sqrt(-2 ln(1 - u2)) cos(2 pi u3) (Box-Muller, in
    // double, rounded to float)
    const uint32_t k0 = (uint32_t)co.seed, k1 = (uint32_t)(co.seed >> 32);
    const U4 r = philox4x32_10(nodes[a].uid, (uint32_t)t, 0u, kApso << 24, k0, k1);
    s_k = (int)__dmul_rn((double)uniform24(r.v[1]), (double)d);
    s_g = (float)__dmul_rn(sqrt(__dmul_rn(-2.0, log((double)__fsub_rn(1.0f, uniform24(r.v[2]))))),
                           cos(__dmul_rn(6.283185307179586, (double)uniform24(r.v[3]))));
  }
  __syncthreads();
  // 3. in the convergence state the next elite candidate: gB with
  // coordinate k moved by (2 sigma) g, sigma = 1 - 0.9 t / T
  if (s_mode) {
    const float sigma = __fsub_rn(1.0f, __fmul_rn(0.9f, __fdiv_rn((float)t, (float)sw.T)));
    for (int j = threadIdx.x; j < d; j += blockDim.x)
      erow[j] = j == s_k ? __fadd_rn(gbp[j], __fmul_rn(__fmul_rn(2.0f, sigma), s_g)) : gbp[j];
  }
  // 4. the move of Eq. pso-1 to iteration t + 1 with the adaptive factors
  // (k_move's step, here by this node's CTA)
  SwarmCoef cm = co;
  cm.inertia = s_c[0];
  cm.c1 = s_c[1];
  cm.c2 = s_c[2];
  const int d4 = (d + 3) >> 2;
  const uint32_t uid = nodes[a].uid;
  for (int item = threadIdx.x; item < P * d4; item += blockDim.x)
    move_item(pr, sw, cm, uid, a, t, item / d4, item - (item / d4) * d4, pbp, gbp);
}

// Algorithm 1's gbest step after evaluation t, then (t < T) the synchronous
// move of Eq. pso-1: every particle moves with the gbest held at the end of
// iteration t. Grid: (node, slice of the node's particle x 4-dimension
// items). Every CTA finds the node's gbest itself; CTA 0 of the node records
// it. The gbest score is double-buffered by iteration parity (read from
// gb[(t-1)&1], written to gb[t&1]) so no CTA reads a score another CTA of
// the launch is writing; the gbest position of a new best is its pbest row.
__global__ void __launch_bounds__(128)
    k_move(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes, int t, SwarmCoef co,
           const int32_t* __restrict__ list, int A) {
  pdl_trigger();
  pdl_wait();
  __shared__ int s_best;
  const int a = list ? list[blockIdx.x] : (int)blockIdx.x;
  const int d = pr.d, d4 = (d + 3) >> 2, Pp = pr.Pp;
  const EvalRes* gold_buf = sw.gb + (int64_t)((t + 1) & 1) * A;
  EvalRes* gnew_buf = sw.gb + (int64_t)(t & 1) * A;
  // with a re-scored subset (sw.sel) k_merge took the gbest step already
  if (!sw.sel && threadIdx.x < 32) {
    const EvalRes gold = gold_buf[a];
    EvalRes be;
    const int bi = gbest_argmin(pr, sw.cur + (int64_t)a * Pp, gold, t, &be);
    if (threadIdx.x == 0) {
      s_best = bi;
      if (blockIdx.y == 0) {
        gnew_buf[a] = bi >= 0 ? be : gold;
        if (bi >= 0) {
          sw.gpart[a] = bi;
          sw.giter[a] = t;
        }
        if (sw.trace) {
          const EvalRes g = bi >= 0 ? be : gold;
          sw.trace[(int64_t)a * (sw.T + 1) + t] =
              g.valid ? g.loss : __longlong_as_double(0x7ff0000000000000LL);
        }
      }
    }
  }
  __syncthreads();
  const int best = sw.sel ? -1 : s_best;
  const float* pbp = sw.pbest + (int64_t)a * Pp * d;
  float* gbp = sw.gbest + (int64_t)a * d;
  // a new best improved its pbest in this iteration: its pbest row is its
  // current position; otherwise the recorded gbest stands
  const float* gsrc = best >= 0 ? pbp + (int64_t)best * d : gbp;
  if (blockIdx.y == 0 && best >= 0)
    for (int j = threadIdx.x; j < d; j += blockDim.x) gbp[j] = gsrc[j];
  if (t >= sw.T) return;
  const uint32_t uid = nodes[a].uid;
  for (int item = blockIdx.y * blockDim.x + threadIdx.x; item < pr.P * d4;
       item += gridDim.y * blockDim.x)
    move_item(pr, sw, co, uid, a, t, item / d4, item % d4, pbp, gsrc);
}

// ---- top-k selection (SLM_PROJ_BF16_TOPK) ------------------------------------------

// ---- histogram and scan -------------------------------------------------------------

constexpr int kCopies = 4;  // histogram copies, each shared by a pair of warps
constexpr int kStages = 2;  // staged pieces: one in flight while one is binned
constexpr int kMseMaxPiece = 2048;  // largest MSE piece (8 entries per thread)

__host__ __device__ inline size_t hist_copy_bytes(int crit, int B, int K) {
  return crit == SLM_MSE ? (size_t)B * (4 + 8 + 8) : (size_t)B * K * 4;
}
// Histogram copies: kCopies shared by warp pairs (classification); one for
// MSE, whose bins are summed by their owner threads after a counting sort.
__host__ __device__ inline int hist_copies(int crit) { return crit == SLM_MSE ? 1 : kCopies; }
// MSE counting-sort scratch: per-bin counts and offsets, the sorted piece.
__host__ __device__ inline size_t sort_bytes(int crit, int B) {
  return crit == SLM_MSE ? (((size_t)(2 * B + 1) * 4 + (size_t)kMseMaxPiece * 2 + 127) & ~(size_t)127)
                         : 0;
}
// Bytes one entry occupies in a stage: z of the particle; the label
// (classification) or the two fixed-point moments (MSE); the multiplicity.
__host__ __device__ inline int entry_bytes(int crit, bool weighted) {
  return (crit == SLM_MSE ? 4 + 8 + 8 : 4 + 4) + (weighted ? 4 : 0);
}
// Entries per staged piece: large pieces (each piece carries fixed costs),
// sized so the stages of two CTAs fit on an SM; a multiple of 256 entries.
__host__ __device__ inline int piece_of(int crit, bool weighted) {
  const int budget = crit == SLM_MSE ? 80 * 1024 : 64 * 1024 + (weighted ? 32 * 1024 : 0);
  return budget / (kStages * entry_bytes(crit, weighted)) / 256 * 256;
}
__host__ __device__ inline size_t stage_bytes(int crit, bool weighted) {
  return (size_t)piece_of(crit, weighted) * entry_bytes(crit, weighted);
}

// A cluster of S CTAs per (node, particle). Rank r streams the r-th of S
// slices of the node's entries through shared memory in pieces: one thread
// issues bulk (TMA) copies of the particle's z, the labels or fixed-point
// moments and the multiplicities of a piece into a ring of kStages stages,
// each with its own mbarrier. Classification: warp w adds its share of a
// piece into histogram copy w % kCopies with shared atomics. MSE: a counting
// sort of the piece by bin, then thread b sums bin b's moments in registers.
// The copies are merged, rank 0 adds the other ranks' histograms through
// distributed shared memory and the whole CTA scans the B-1 edges. In a
// search (do_update) rank 0 also takes the particle's pbest step; the gbest
// step and the move follow in k_move.
__global__ void __launch_bounds__(kThreads, 3)
    k_hist_scan(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes,
                const int32_t* __restrict__ list, int32_t* bins_out, int t, int do_update) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar[kStages];
  __shared__ int s_ok;
  __shared__ float s_zmin, s_inv_w;
  __shared__ ScanScratch sc;
  const cg::cluster_group cl = cg::this_cluster();
  pdl_trigger();
  pdl_wait();
  const int S = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int a = list ? list[blockIdx.x / S] : (int)blockIdx.x / S;
  const int p = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const NodeDesc nd = nodes[a];
  const int B = pr.B, K = pr.K;
  const bool mse = pr.crit == SLM_MSE;
  const bool weighted = pr.w != nullptr;
  const int words = mse ? B : B * K;  // u32 counters per copy
  const int piece = piece_of(pr.crit, weighted);
  // shared memory: the histogram copies, the MSE sort scratch, two stages.
  // MSE bins hold the weight and the fixed-point sums of w (y-c) and w (y-c)^2.
  const int ncopies = hist_copies(pr.crit);
  unsigned long long* hs = reinterpret_cast<unsigned long long*>(smem);  // MSE [B]
  unsigned long long* hq = hs + (mse ? B : 0);                            // MSE [B]
  uint32_t* hc = reinterpret_cast<uint32_t*>(hq + (mse ? B : 0));  // [ncopies][words]
  unsigned char* sort0 =
      smem + ((hist_copy_bytes(pr.crit, B, K) * ncopies + 127) & ~(size_t)127);
  uint32_t* pcnt = reinterpret_cast<uint32_t*>(sort0);  // MSE [B] entries per bin of a piece
  uint32_t* poff = pcnt + B;                            // MSE [B + 1] their offsets
  uint16_t* sorted = reinterpret_cast<uint16_t*>(poff + B + 1);  // MSE [piece]
  unsigned char* stage0 = sort0 + sort_bytes(pr.crit, B);
  const size_t sbytes = stage_bytes(pr.crit, weighted);
  const int copy = warp % ncopies;
  uint32_t* h = hc + copy * words;

  int* zz = sw.zmm + ((int64_t)a * pr.Pp + p) * 2;
  if (threadIdx.x == 0) {
    const int lo_o = zz[0], hi_o = zz[1];
    float zmin = 0.f, inv_w = 0.f;
    int ok = 0;
    if (lo_o != INT_MAX) {
      const float lo = ord2f(lo_o), hi = ord2f(hi_o);
      inv_w = __fdiv_rn((float)B, __fsub_rn(hi, lo));
      zmin = lo;
      ok = (hi > lo) && isfinite(inv_w);
    }
    s_zmin = zmin;
    s_inv_w = inv_w;
    s_ok = ok;
    for (int i = 0; i < kStages; ++i) mbar_init(&s_bar[i], 1);
    mbar_init_fence();
  }
  for (int i = threadIdx.x; i < ncopies * words; i += kThreads) hc[i] = 0u;
  if (mse)
    for (int i = threadIdx.x; i < B; i += kThreads) {
      hs[i] = 0ull;
      hq[i] = 0ull;
      pcnt[i] = 0u;
    }
  __syncthreads();
  const bool ok = s_ok;
  const float zmin = s_zmin, inv_w = s_inv_w;

  // slice of this rank: starts on a multiple of 4 entries (16 bytes)
  const int chunk = ((nd.seg_len + S - 1) / S + 3) & ~3;
  const int r_begin = min(nd.seg_len, rank * chunk);
  const int r_end = min(nd.seg_len, r_begin + chunk);
  const int n_pieces = ok ? (r_end - r_begin + piece - 1) / piece : 0;
  const int64_t e0 = nd.seg_start;  // multiple of 4
  // stage layout: z [piece] f32 | labels [piece] i32, or moments 2 x [piece]
  // i64 | multiplicities [piece] u32
  const size_t off_w = (size_t)piece * (mse ? 4 + 16 : 4 + 4);
  auto issue = [&](int k) {
    const int r = r_begin + k * piece;
    const int n = min(piece, r_end - r);
    const uint32_t bytes = (uint32_t)(((n + 3) & ~3) * 4);
    unsigned char* st = stage0 + (k % kStages) * sbytes;
    uint64_t* bar = &s_bar[k % kStages];
    fence_proxy_async();
    mbar_expect_tx(bar, bytes * (uint32_t)((mse ? 5 : 2) + (weighted ? 1 : 0)));
    bulk_g2s(st, sw.z + (int64_t)p * pr.Ez + e0 + r, bytes, bar);
    if (mse) {
      bulk_g2s(st + (size_t)piece * 4, pr.m1 + e0 + r, 2 * bytes, bar);
      bulk_g2s(st + (size_t)piece * 12, pr.m2 + e0 + r, 2 * bytes, bar);
    } else {
      bulk_g2s(st + (size_t)piece * 4, pr.lab + e0 + r, bytes, bar);
    }
    if (weighted) bulk_g2s(st + off_w, pr.w + e0 + r, bytes, bar);
  };
  unsigned long long acc1 = 0ull, acc2 = 0ull;  // MSE: bin threadIdx.x of this slice
  uint32_t accw = 0u;
  if (threadIdx.x == 0)
    for (int k = 0; k < kStages - 1 && k < n_pieces; ++k) issue(k);
  for (int k = 0; k < n_pieces; ++k) {
    // piece k + kStages - 1 reuses the stage of piece k - 1, released by the
    // barrier at the end of the previous round
    if (threadIdx.x == 0 && k + kStages - 1 < n_pieces) issue(k + kStages - 1);
    const uint32_t parity = (uint32_t)((k / kStages) & 1);
    if (!mbar_wait(&s_bar[k % kStages], parity, d_first_wait_polls)) {
      // a copy did not land: record it, give the copies in flight a bounded
      // chance to finish, and stop using the stages
      if (threadIdx.x == 0 && sw.err) atomicExch(sw.err, kErrCopyTimeout);
      for (int j = k; j < n_pieces && j < k + kStages; ++j)
        mbar_wait(&s_bar[j % kStages], (uint32_t)((j / kStages) & 1), kWaitPolls);
      break;
    }
    const unsigned char* st = stage0 + (k % kStages) * sbytes;
    const int r = r_begin + k * piece;
    const int n = min(piece, r_end - r);
    const float* zs = reinterpret_cast<const float*>(st);
    const int32_t* ls = reinterpret_cast<const int32_t*>(st + (size_t)piece * 4);
    const unsigned long long* m1s =
        reinterpret_cast<const unsigned long long*>(st + (size_t)piece * 4);
    const unsigned long long* m2s =
        reinterpret_cast<const unsigned long long*>(st + (size_t)piece * 12);
    const uint32_t* ws = reinterpret_cast<const uint32_t*>(st + off_w);
    if (mse) {
      // counting sort of the piece by bin (slot = arrival order in the bin),
      // then thread b sums bin b's moments in registers: no 64-bit atomics
      int bb[kMseMaxPiece / kThreads], sl[kMseMaxPiece / kThreads];
#pragma unroll
      for (int u = 0; u < kMseMaxPiece / kThreads; ++u) {
        const int i = threadIdx.x + u * kThreads;
        bb[u] = -1;
        if (i < n) {
          const int b = bin_of(zs[i], zmin, inv_w, B);
          bb[u] = b;
          sl[u] = (int)atomicAdd(&pcnt[b], 1u);
          if (bins_out) bins_out[(int64_t)p * nd.seg_len + r + i] = b;
        }
      }
      __syncthreads();
      if (warp == 0) {  // exclusive prefix of the counts
        const int bpl = (B + 31) >> 5;
        uint32_t sum = 0;
        for (int q = 0; q < bpl; ++q) {
          const int j = lane * bpl + q;
          if (j < B) sum += pcnt[j];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const uint32_t v = __shfl_up_sync(0xffffffffu, inc, off);
          if (lane >= off) inc += v;
        }
        uint32_t run = inc - sum;
        for (int q = 0; q < bpl; ++q) {
          const int j = lane * bpl + q;
          if (j < B) {
            poff[j] = run;
            run += pcnt[j];
          }
        }
        if (lane == 31) poff[B] = inc;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < kMseMaxPiece / kThreads; ++u)
        if (bb[u] >= 0) sorted[poff[bb[u]] + sl[u]] = (uint16_t)(threadIdx.x + u * kThreads);
      __syncthreads();
      if ((int)threadIdx.x < B) {
        const int b = threadIdx.x;
        const int j1 = (int)poff[b + 1];
        for (int j = (int)poff[b]; j < j1; ++j) {
          const int i = sorted[j];
          acc1 += m1s[i];  // two's complement: signed sums wrap exactly
          acc2 += m2s[i];
          accw += weighted ? ws[i] : 1u;
        }
        pcnt[b] = 0u;
      }
    } else {
      for (int i = threadIdx.x; i < n; i += kThreads) {
        const int b = bin_of(zs[i], zmin, inv_w, B);
        const uint32_t w = weighted ? ws[i] : 1u;
        atomicAdd(&h[b * K + ls[i]], w);
        if (bins_out) bins_out[(int64_t)p * nd.seg_len + r + i] = b;
      }
    }
    __syncthreads();  // this stage is refilled by piece k + kStages
  }
  if (mse && (int)threadIdx.x < B) {  // the owner threads' bins
    hc[threadIdx.x] = accw;
    hs[threadIdx.x] = acc1;
    hq[threadIdx.x] = acc2;
  }
  // merge the warp copies into copy 0
  if (ncopies > 1) {
    __syncthreads();
    for (int i = threadIdx.x; i < words; i += kThreads) {
      uint32_t v = 0;
#pragma unroll
      for (int c = 0; c < kCopies; ++c) v += hc[c * words + i];
      hc[i] = v;
    }
  }
  if (S > 1) {
    cl.sync();  // every rank's copy 0 is complete
    if (rank == 0) {
      for (int i = threadIdx.x; i < words; i += kThreads) {
        uint32_t v = hc[i];
#pragma unroll
        for (int q = 1; q < 16; ++q)
          if (q < S) v += cl.map_shared_rank(hc, q)[i];
        hc[i] = v;
      }
      if (mse)
        for (int i = threadIdx.x; i < B; i += kThreads) {
          unsigned long long vs = hs[i], vq = hq[i];
          for (int q = 1; q < S; ++q) {
            vs += cl.map_shared_rank(hs, q)[i];
            vq += cl.map_shared_rank(hq, q)[i];
          }
          hs[i] = vs;
          hq[i] = vq;
        }
    }
    cl.sync();  // the other ranks' memory is no longer read
    if (rank != 0) return;
  }
  __syncthreads();
  EvalRes res;
  if (!ok) {
    res = invalid_res();
  } else {
    res = mse ? block_scan_mse(hc, reinterpret_cast<const long long*>(hs),
                               reinterpret_cast<const long long*>(hq), pr.mscale[2 * a],
                               pr.mscale[2 * a + 1], B, pr.min_leaf, sc)
              : pr.crit == SLM_GINI ? block_scan_cls<SLM_GINI>(hc, B, K, pr.min_leaf, sc)
                                    : block_scan_cls<SLM_ENTROPY>(hc, B, K, pr.min_leaf, sc);
    res.zmin = zmin;
    res.inv_w = inv_w;
  }
  if (threadIdx.x == 0) {
    sw.cur[(int64_t)a * pr.Pp + p] = res;
    zz[0] = INT_MAX;  // ready for the next iteration
    zz[1] = INT_MIN;
    if (do_update) mark_improvement(pr, sw, a, t, res);
  }
  if (do_update && warp == 0) {
    pbest_step(pr, sw, a, p, t, res);
    if (sw.ic && t < sw.T) {
      __syncwarp();  // the pbest row the lanes just wrote
      premove_particle(pr, sw, nd.uid, a, t, p);
    }
  }
  if (sw.tk_sel) {
    // the last particle of the node to be scored selects the node's top k
    __shared__ int s_last;
    __threadfence();  // this CTA's score write before the count
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&sw.done[a], 1) == pr.P - 1;
    __syncthreads();
    if (s_last) {
      __threadfence();
      topk_select(pr, sw, a, stage0);  // the stages are free by now
      if (threadIdx.x == 0) sw.done[a] = 0;
    }
  }
}

// Classification threshold scan of one particle by one warp: the arithmetic
// and tie rules of block_scan_cls (per-class prefix over bins, per-edge
// counts, Gini rational or entropy loss, repeated partitions skipped, lower
// edge on ties), so the same score. h: [B][K] counts (prefix sums in place).
template <int CRIT>
__device__ EvalRes warp_scan_cls(uint32_t* h, int B, int K, int min_leaf) {
  const int lane = threadIdx.x & 31;
  const int bpl = (B + 31) >> 5;
  for (int k = 0; k < K; ++k) {
    uint32_t v[kMaxBins / 32];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kMaxBins / 32; ++i) {
      const int j = lane * bpl + i;
      v[i] = (i < bpl && j < B) ? h[j * K + k] : 0u;
      sum += v[i];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += u;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int i = 0; i < kMaxBins / 32; ++i) {
      const int j = lane * bpl + i;
      run += v[i];
      if (i < bpl && j < B) h[j * K + k] = run;
    }
  }
  __syncwarp();
  const uint32_t* tot = h + (B - 1) * K;
  uint32_t ntot = 0;
  for (int k = 0; k < K; ++k) ntot += tot[k];
  uint64_t bn = 0, bd = 0;
  double bl = 0.0;
  int bb = -1;
  uint32_t bnl = 0;
  for (int b = 1 + lane; b < B; b += 32) {
    const uint32_t* row = h + (b - 1) * K;
    uint32_t nl = 0, prev = 0;
    for (int k = 0; k < K; ++k) {
      nl += row[k];
      if (b >= 2) prev += row[k - K];
    }
    const uint32_t nr = ntot - nl;
    // only an admissible edge is scored (the c ln c terms are table reads)
    if (nl != prev && nl >= (uint32_t)min_leaf && nr >= (uint32_t)min_leaf) {
      uint64_t cn = 0, cd = 0;
      double cl = 0.0;
      if (CRIT == SLM_GINI) {
        uint64_t sl = 0, sr = 0;
        for (int k = 0; k < K; ++k) {
          const uint32_t l = row[k], r = tot[k] - l;
          sl += (uint64_t)l * l;
          sr += (uint64_t)r * r;
        }
        cn = sl * nr + sr * nl;
        cd = (uint64_t)nl * nr;
      } else {
        // the class terms summed in class order, several table reads in flight
        const double tl = xlogx_t(nl), tr = xlogx_t(nr);
        double hl = 0.0, hr = 0.0;
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
          const uint32_t l = row[k], r = tot[k] - l;
          hl += xlogx_t(l);
          hr += xlogx_t(r);
        }
        cl = ((tl - hl) + (tr - hr)) / (double)ntot;
      }
      if (edge_takes<CRIT>(cn, cd, cl, b, bn, bd, bl, bb)) {
        bn = cn;
        bd = cd;
        bl = cl;
        bb = b;
        bnl = nl;
      }
    }
  }
  // the warp argmin on a 32-bit key of each lane's best loss (one warp
  // reduction), the lanes within 8 ulps of the smallest key compared
  // exactly in lane order (= edge order within each lane's stride): the
  // key's rounding is far below 8 ulps, so the choice is the exact one
  uint32_t key = 0xffffffffu;
  if (bb >= 0) {
    float lf;
    if (CRIT == SLM_GINI) {
      const uint64_t nden = (uint64_t)ntot * bd;
      lf = __fdiv_rn((float)(nden - bn), (float)nden);
    } else {
      lf = (float)bl;
    }
    const uint32_t u = __float_as_uint(lf);
    key = (u >> 31) ? ~u : (u | 0x80000000u);  // the float order as unsigned
  }
  {
    const uint32_t kmin = __reduce_min_sync(0xffffffffu, key);
    unsigned m = __ballot_sync(0xffffffffu, bb >= 0 && key - kmin <= 8u);
    int wi = m ? __ffs(m) - 1 : 0;
    uint64_t wn = __shfl_sync(0xffffffffu, bn, wi), wd = __shfl_sync(0xffffffffu, bd, wi);
    double wl = __shfl_sync(0xffffffffu, bl, wi);
    int wb = m ? __shfl_sync(0xffffffffu, bb, wi) : -1;
    uint32_t wnl = __shfl_sync(0xffffffffu, bnl, wi);
    m = m ? m & (m - 1) : 0u;
    while (m) {  // rare: several lanes within a few ulps
      const int li = __ffs(m) - 1;
      m &= m - 1;
      const uint64_t on = __shfl_sync(0xffffffffu, bn, li), od = __shfl_sync(0xffffffffu, bd, li);
      const double ol = __shfl_sync(0xffffffffu, bl, li);
      const int ob = __shfl_sync(0xffffffffu, bb, li);
      const uint32_t onl = __shfl_sync(0xffffffffu, bnl, li);
      if (edge_takes<CRIT>(on, od, ol, ob, wn, wd, wl, wb)) {
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
  }
  EvalRes res = invalid_res();
  if (bb >= 0) {
    res.valid = 1;
    res.bin = bb;
    res.nl = bnl;
    res.nr = ntot - bnl;
    if (CRIT == SLM_GINI) {
      res.num = bn;
      res.den = bd;
      const uint64_t nden = (uint64_t)ntot * res.den;
      res.loss = (double)(nden - res.num) / (double)nden;
    } else {
      res.loss = bl;
    }
  }
  return res;
}

// Histogram and threshold scan of the particles of small classification
// nodes (list[]: their indices), one warp per (node, particle): the warp
// reads the node's z and labels (and multiplicities) straight from memory
// (L2-resident at these sizes) into its own shared histogram and scans it
// with warp_scan_cls. The score, the range reset and the pbest step are
// those of k_hist_scan; small nodes save its per-CTA staging, copies,
// merges and block-wide barriers.
template <int CRIT>
__global__ void __launch_bounds__(kThreads)
    k_hist_warp(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes,
                const int32_t* __restrict__ list, int n_pairs, int t, int do_update) {
  extern __shared__ __align__(16) uint32_t hw[];
  pdl_trigger();
  pdl_wait();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q = (int)blockIdx.x * (kThreads / 32) + warp;
  if (q >= n_pairs) return;  // the whole warp
  const int a = list[q / pr.P], p = q % pr.P;
  const NodeDesc nd = nodes[a];
  const int B = pr.B, K = pr.K, words = B * K;
  uint32_t* h = hw + warp * words;
  int* zz = sw.zmm + ((int64_t)a * pr.Pp + p) * 2;
  const int lo_o = zz[0], hi_o = zz[1];
  float zmin = 0.f, inv_w = 0.f;
  bool ok = false;
  if (lo_o != INT_MAX) {
    const float lo = ord2f(lo_o), hi = ord2f(hi_o);
    inv_w = __fdiv_rn((float)B, __fsub_rn(hi, lo));
    zmin = lo;
    ok = (hi > lo) && isfinite(inv_w);
  }
  for (int i = lane; i < words; i += 32) h[i] = 0u;
  __syncwarp();
  if (ok) {
    const float* zs = sw.z + (int64_t)p * pr.Ez + nd.seg_start;
    const int32_t* ls = pr.lab + nd.seg_start;
    const uint32_t* ws = pr.w ? pr.w + nd.seg_start : nullptr;
    const int n = nd.seg_len;
    int done = 0;
    if (((reinterpret_cast<uintptr_t>(zs) | reinterpret_cast<uintptr_t>(ls) |
          reinterpret_cast<uintptr_t>(ws)) & 15) == 0) {
      // sixteen entries per lane in flight (four 16-byte groups of z, labels
      // and multiplicities) before their shared atomics: the node's z has
      // often left L2 by now, and each round trip is then a DRAM one
      constexpr int U = 4;
      const int n4 = n >> 2;
      for (int g0 = lane; g0 < n4; g0 += 32 * U) {
        float4 zv[U];
        int4 lv[U];
        uint4 wv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int g = g0 + 32 * u;
          const bool in = g < n4;
          zv[u] = in ? __ldcg(reinterpret_cast<const float4*>(zs) + g) : make_float4(0, 0, 0, 0);
          lv[u] = in ? __ldg(reinterpret_cast<const int4*>(ls) + g) : make_int4(-1, -1, -1, -1);
          wv[u] = in && ws ? __ldg(reinterpret_cast<const uint4*>(ws) + g) : make_uint4(1, 1, 1, 1);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (lv[u].x < 0) continue;  // past the node (whole group)
          atomicAdd(&h[bin_of(zv[u].x, zmin, inv_w, B) * K + lv[u].x], wv[u].x);
          atomicAdd(&h[bin_of(zv[u].y, zmin, inv_w, B) * K + lv[u].y], wv[u].y);
          atomicAdd(&h[bin_of(zv[u].z, zmin, inv_w, B) * K + lv[u].z], wv[u].z);
          atomicAdd(&h[bin_of(zv[u].w, zmin, inv_w, B) * K + lv[u].w], wv[u].w);
        }
      }
      done = n4 << 2;
    }
    // the rest (or every entry where the arrays are not 16-byte aligned),
    // four per lane in flight
    for (int i0 = done + lane; i0 < n; i0 += 128) {
      float zv[4];
      int32_t lv[4];
      uint32_t wv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + 32 * u;
        const bool in = i < n;
        zv[u] = in ? __ldcg(zs + i) : 0.f;
        lv[u] = in ? __ldg(ls + i) : -1;
        wv[u] = in && ws ? __ldg(ws + i) : 1u;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (lv[u] >= 0) atomicAdd(&h[bin_of(zv[u], zmin, inv_w, B) * K + lv[u]], wv[u]);
    }
  }
  __syncwarp();
  EvalRes res = invalid_res();
  if (ok) {
    res = warp_scan_cls<CRIT>(h, B, K, pr.min_leaf);
    res.zmin = zmin;
    res.inv_w = inv_w;
  }
  if (lane == 0) {
    sw.cur[(int64_t)a * pr.Pp + p] = res;
    zz[0] = INT_MAX;  // ready for the next iteration
    zz[1] = INT_MIN;
    if (do_update) mark_improvement(pr, sw, a, t, res);
  }
  if (do_update) {
    pbest_step(pr, sw, a, p, t, res);
    if (sw.ic && t < sw.T) {
      __syncwarp();  // the pbest row the lanes just wrote
      premove_particle(pr, sw, nd.uid, a, t, p);
    }
  }
}

// Persistent search of small classification nodes: all T + 1 iterations of
// Algorithm 1 in one launch, the swarm kept on chip. A cluster of S CTAs per
// node (grid (S, nodes)); rank r owns the particle groups g = r, r + S, ...
// (particles 8g .. 8g+7) and keeps their positions, velocities, pbest rows
// and pbest scores in its shared memory for the whole search, with the
// node's rows, labels and multiplicities. Per group, the whole CTA projects
// the group's 8 particles onto every row (each thread 4 rows x 8 particles
// in registers; rows as 16-byte chunks, XOR-swizzled so that lanes on
// consecutive rows read distinct banks; every z is the sequential fused
// multiply-add over the features of k_project) into a shared z buffer,
// folding in each particle's exact range; warps 2j and 2j+1 bin particle
// 8g + j's halves of the rows into its histogram, warp 2j runs warp_scan_cls (the scores of the per-iteration kernels) and takes the
// pbest step in shared memory. After a cluster barrier every CTA gathers all
// particles' scores through distributed shared memory and takes the gbest
// step of k_move (the same argmin, the same gold), reads a new gB row from
// its owner's pbest rows, and moves its own particles with move_item's
// arithmetic and draws; a second barrier keeps scores and pbest rows from
// being rewritten while other CTAs read them. The search's results (gbest
// score, particle, iteration and row, trace, and each particle's final
// position, velocity, pbest and score) go to global memory with the
// per-iteration kernels' layout and meaning. d must be a multiple of 4.

// Position in a row of 16-byte chunk c (C chunks per row) of row r: rows r
// .. r+7 then fall in distinct bank groups.
__device__ __forceinline__ int node_chunk(int r, int c, int C) {
  const int x = (C & 1) ? 0 : (C & 3) == 2 ? (r >> 2) & 1 : (C & 7) == 4 ? (r >> 1) & 3 : r & 7;
  return c ^ x;
}

// Words of one score record (copied between shared memories word by word).
constexpr int kResWords = (int)(sizeof(EvalRes) / 4);

// Particle slots a CTA of an S-CTA cluster owns: 8 per owned group.
__host__ __device__ inline int node_search_slots(int P, int S) {
  return 8 * ((((P + 7) >> 3) + S - 1) / S);
}

template <int CRIT>
__global__ void __launch_bounds__(kNodeThreads)
    k_node_search(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes,
                  const int32_t* __restrict__ list, int A, SwarmCoef co) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) float nsm[];
  __shared__ int s_best;
  __shared__ int s_lo[8], s_hi[8];
  __shared__ EvalRes s_gold;  // the gbest score after the last evaluation
  __shared__ int s_gpart, s_giter;
  const cg::cluster_group cl = cg::this_cluster();
  pdl_trigger();
  pdl_wait();
  const int S = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int a = list[blockIdx.y];
  const NodeDesc nd = nodes[a];
  const int n = nd.seg_len, d = pr.d, C = d >> 2, B = pr.B, K = pr.K, P = pr.P, Pp = pr.Pp;
  const int d4 = (d + 3) >> 2;
  const bool weighted = pr.w != nullptr;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_groups = (P + 7) >> 3;
  const int my_groups = rank < n_groups ? (n_groups - 1 - rank) / S + 1 : 0;
  // shared memory (node_search_smem; d is a multiple of 4, so every
  // float array starts on 16 bytes): rows, z, the owned particles' state
  // (8 per owned group), gB, scores, histograms, labels, multiplicities
  float* xs = nsm;                                             // [n][d], swizzled chunks
  float* zb = xs + (size_t)n * d;                              // [8][n]
  const int slots = node_search_slots(P, S);                  // owned particle slots
  float* ppos = zb + (size_t)8 * n;                            // [slots][d]
  float* pvel = ppos + (size_t)slots * d;                      // [slots][d]
  float* ppb = pvel + (size_t)slots * d;                       // [slots][d] pbest rows
  float* gbr = ppb + (size_t)slots * d;                        // [d] gB
  EvalRes* spb = reinterpret_cast<EvalRes*>(gbr + d);          // [slots] pbest scores
  EvalRes* scur = spb + slots;                                 // [slots] this evaluation's
  EvalRes* sall = scur + slots;                                // [P] every particle's
  uint32_t* hist = reinterpret_cast<uint32_t*>(sall + P);      // [8][B * K]
  int32_t* ls = reinterpret_cast<int32_t*>(hist + 8 * B * K);   // [n]
  uint32_t* wsm = reinterpret_cast<uint32_t*>(ls + n);          // [n] (weighted)
  const int64_t e0 = nd.seg_start;
  const int64_t nb = (int64_t)a * Pp;  // the node's first particle row
  // owned slot s = 8 (group / S) + (p mod 8) of particle p in group g = p / 8
  auto owner = [&](int p) { return (p >> 3) % S; };
  auto slot = [&](int p) { return ((p >> 3) / S) * 8 + (p & 7); };
  for (int q = threadIdx.x; q < n * C; q += kNodeThreads) {
    const int r = q / C, c = q - r * C;
    *reinterpret_cast<float4*>(xs + (size_t)r * d + 4 * node_chunk(r, c, C)) =
        *reinterpret_cast<const float4*>(pr.X + (e0 + r) * d + 4 * c);
  }
  for (int i = threadIdx.x; i < n; i += kNodeThreads) {
    ls[i] = pr.lab[e0 + i];
    if (weighted) wsm[i] = pr.w[e0 + i];
  }
  // the owned particles' start (zero rows past P stay zero: they project to 0)
  for (int q = threadIdx.x; q < my_groups * 8 * d; q += kNodeThreads) {
    const int sl = q / d, k = q - sl * d;
    const int p = 8 * (rank + (sl >> 3) * S) + (sl & 7);
    const bool in = p < P;
    ppos[q] = in ? sw.pos[(nb + p) * d + k] : 0.0f;
    pvel[q] = in ? sw.vel[(nb + p) * d + k] : 0.0f;
    ppb[q] = 0.0f;
  }
  if (threadIdx.x == 0) {
    s_gold = invalid_res();
    s_gpart = 0;
    s_giter = 0;
  }
  __syncthreads();
  const int j = warp >> 1, half = warp & 1;  // particle of the group, half of the rows
  uint32_t* h = hist + j * B * K;            // particle j's histogram (both halves add in)
  for (int t = 0; t <= sw.T; ++t) {
    for (int lg = 0; lg < my_groups; ++lg) {
      const int g = rank + lg * S;
      const float* apos = ppos + (size_t)lg * 8 * d;  // the group's positions, [8][d]
      if (threadIdx.x < 8) {
        s_lo[threadIdx.x] = INT_MAX;
        s_hi[threadIdx.x] = INT_MIN;
      }
      for (int i = threadIdx.x; i < 8 * B * K; i += kNodeThreads) hist[i] = 0u;
      __syncthreads();
      // z of the group's 8 particles on every row, 4 rows per thread at once;
      // the exact range of each particle folded in as ordered integers
      int lo_t[8], hi_t[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        lo_t[jj] = INT_MAX;
        hi_t[jj] = INT_MIN;
      }
      for (int r0 = threadIdx.x; r0 < n; r0 += 4 * kNodeThreads) {
        float acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) acc[i][jj] = 0.0f;
        for (int c = 0; c < C; ++c) {
          float4 xv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int r = r0 + i * kNodeThreads;
            xv[i] = r < n ? *reinterpret_cast<const float4*>(xs + (size_t)r * d +
                                                             4 * node_chunk(r, c, C))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
          }
          // feature by feature over all 32 accumulators: each accumulator
          // still takes the chunk's features in increasing order
          float4 pv[8];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
            pv[jj] = *reinterpret_cast<const float4*>(apos + jj * d + 4 * c);
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i][jj] = fmaf(xv[i].x, pv[jj].x, acc[i][jj]);
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i][jj] = fmaf(xv[i].y, pv[jj].y, acc[i][jj]);
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i][jj] = fmaf(xv[i].z, pv[jj].z, acc[i][jj]);
#pragma unroll
          for (int jj = 0; jj < 8; ++jj)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[i][jj] = fmaf(xv[i].w, pv[jj].w, acc[i][jj]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = r0 + i * kNodeThreads;
          if (r < n)
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              zb[(size_t)jj * n + r] = acc[i][jj];
              const int o = f2ord(acc[i][jj]);
              lo_t[jj] = min(lo_t[jj], o);
              hi_t[jj] = max(hi_t[jj], o);
            }
        }
      }
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int lo = __reduce_min_sync(0xffffffffu, lo_t[jj]);
        const int hi = __reduce_max_sync(0xffffffffu, hi_t[jj]);
        if (lane == 0 && lo != INT_MAX) {
          atomicMin(&s_lo[jj], lo);
          atomicMax(&s_hi[jj], hi);
        }
      }
      __syncthreads();
      const int p = 8 * g + j;
      float zmin = 0.f, inv_w = 0.f;
      bool ok = false;
      if (s_lo[j] != INT_MAX) {
        const float lo = ord2f(s_lo[j]), hi = ord2f(s_hi[j]);
        inv_w = __fdiv_rn((float)B, __fsub_rn(hi, lo));
        zmin = lo;
        ok = (hi > lo) && isfinite(inv_w);
      }
      if (ok && p < P) {
        // this warp's half of the rows into the particle's histogram, four
        // entries per lane in flight
        const float* zp = zb + (size_t)j * n;
        for (int r0 = half * 32 + lane; r0 < n; r0 += 256) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = r0 + 64 * u;
            if (r < n)
              atomicAdd(&h[bin_of(zp[r], zmin, inv_w, B) * K + ls[r]], weighted ? wsm[r] : 1u);
          }
        }
      }
      __syncthreads();
      if (half == 0 && p < P) {
        EvalRes res = invalid_res();
        if (ok) {
          res = warp_scan_cls<CRIT>(h, B, K, pr.min_leaf);
          res.zmin = zmin;
          res.inv_w = inv_w;
        }
        // the score, and the pbest step (Algorithm 1: strict "<"; the
        // position is kept on improvement) in shared memory
        const int sl = lg * 8 + j;
        int imp = 0;
        if (lane == 0) {
          scur[sl] = res;
          imp = (t == 0) || better(res, spb[sl], pr.crit);
          if (imp) spb[sl] = res;
        }
        imp = __shfl_sync(0xffffffffu, imp, 0);
        if (imp)
          for (int k = lane; k < d; k += 32) ppb[(size_t)sl * d + k] = ppos[(size_t)sl * d + k];
      }
      __syncthreads();  // zb, ranges and histograms are reset for the next group
    }
    // every CTA's scores and pbest rows of evaluation t are in place
    cl.sync();
    // every particle's score, in particle order, from its owner
    for (int q = threadIdx.x; q < P * kResWords; q += kNodeThreads) {
      const int pp = q / kResWords, w = q - pp * kResWords;
      const uint32_t* src = reinterpret_cast<const uint32_t*>(
          cl.map_shared_rank(scur + slot(pp), owner(pp)));
      reinterpret_cast<uint32_t*>(sall + pp)[w] = src[w];
    }
    __syncthreads();
    // gbest step (k_move's rule: the argmin against the gbest of the last
    // evaluation, every particle a candidate at evaluation 0)
    if (warp == 0) {
      const EvalRes gold = s_gold;
      EvalRes be;
      const int bi = gbest_argmin(pr, sall, gold, t, &be);
      if (lane == 0) {
        s_best = bi;
        if (bi >= 0) {
          s_gold = be;
          s_gpart = bi;
          s_giter = t;
        }
        if (rank == 0 && sw.trace) {
          const EvalRes gr = bi >= 0 ? be : gold;
          sw.trace[(int64_t)a * (sw.T + 1) + t] =
              gr.valid ? gr.loss : __longlong_as_double(0x7ff0000000000000LL);
        }
      }
    }
    __syncthreads();
    const int best = s_best;
    // a new best improved its pbest in this evaluation: gB is that row
    if (best >= 0) {
      const float* src = cl.map_shared_rank(ppb + (size_t)slot(best) * d, owner(best));
      for (int k = threadIdx.x; k < d; k += kNodeThreads) gbr[k] = src[k];
    }
    __syncthreads();
    if (t < sw.T) {
      // the owned particles' move (move_item's draws and roundings)
      const uint32_t k0 = (uint32_t)co.seed, k1 = (uint32_t)(co.seed >> 32);
      for (int item = threadIdx.x; item < my_groups * 8 * d4; item += kNodeThreads) {
        const int sl = item / d4, q = item - sl * d4;
        const int pi = 8 * (rank + (sl >> 3) * S) + (sl & 7);
        if (pi >= P) continue;
        const U4 r1 = philox4x32_10(nd.uid, (uint32_t)(t + 1), (uint32_t)pi,
                                    (uint32_t)q | (kR1 << 24), k0, k1);
        const U4 r2 = philox4x32_10(nd.uid, (uint32_t)(t + 1), (uint32_t)pi,
                                    (uint32_t)q | (kR2 << 24), k0, k1);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int k = 4 * q + c;
          if (k >= d) break;
          const size_t o = (size_t)sl * d + k;
          const float x = ppos[o], v = pvel[o];
          const float inertia = __fmul_rn(co.inertia, v);
          const float cog =
              __fmul_rn(__fmul_rn(co.c1, uniform24(r1.v[c])), __fsub_rn(ppb[o], x));
          const float soc = __fmul_rn(__fmul_rn(co.c2, uniform24(r2.v[c])), __fsub_rn(gbr[k], x));
          const float vn = __fadd_rn(__fadd_rn(inertia, cog), soc);
          pvel[o] = vn;
          ppos[o] = __fadd_rn(x, vn);
        }
      }
    }
    // no score or pbest row is rewritten while another CTA may read it
    cl.sync();
  }
  // the search's results, with the per-iteration kernels' layout
  for (int q = threadIdx.x; q < my_groups * 8 * d; q += kNodeThreads) {
    const int sl = q / d, k = q - sl * d;
    const int p = 8 * (rank + (sl >> 3) * S) + (sl & 7);
    if (p >= P) continue;
    sw.pos[(nb + p) * d + k] = ppos[q];
    sw.vel[(nb + p) * d + k] = pvel[q];
    sw.pbest[(nb + p) * d + k] = ppb[q];
  }
  for (int sl = threadIdx.x; sl < my_groups * 8; sl += kNodeThreads) {
    const int p = 8 * (rank + (sl >> 3) * S) + (sl & 7);
    if (p >= P) continue;
    sw.pb[nb + p] = spb[sl];
    sw.cur[nb + p] = scur[sl];
  }
  if (rank == 0) {
    for (int k = threadIdx.x; k < d; k += kNodeThreads) sw.gbest[(int64_t)a * d + k] = gbr[k];
    if (threadIdx.x == 0) {
      sw.gb[(int64_t)(sw.T & 1) * A + a] = s_gold;
      sw.gpart[a] = s_gpart;
      sw.giter[a] = s_giter;
    }
  }
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
  if (sw.posb) {  // the positions as bfloat16 MMA operands, padding zero
    __syncthreads();
    const int dp4 = pr.dp >> 2;
    for (int e = threadIdx.x; e < pr.Pp * dp4; e += blockDim.x) {
      const int p = e / dp4, j0 = 4 * (e - p * dp4);
      float v[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] = j0 + c < d ? pos[(int64_t)p * d + j0 + c] : 0.0f;
      store_posb4(sw.posb, pr.Pp, pr.dp, a, p, j0, v);
    }
  }
  if (threadIdx.x == 0) {
    sw.gb[a] = invalid_res();
    sw.gb[gridDim.x + a] = invalid_res();
    sw.gpart[a] = 0;
    sw.giter[a] = 0;
    if (sw.apso) sw.apso[a] = ApsoState{1, 0, co.c1, co.c2, co.inertia};
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

// ---- MSE moments ------------------------------------------------------------------

__global__ void k_mse_init(int A, unsigned long long* acc_w, int32_t* acc_y) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A) return;
  acc_w[a] = 0ull;
  acc_y[2 * a] = INT_MAX;
  acc_y[2 * a + 1] = INT_MIN;
}

// One CTA per kTS-row tile: the tile's weight and range of y, folded into its node.
__global__ void __launch_bounds__(kTS)
    k_mse_range(Problem pr, const WorkTile* __restrict__ tiles, unsigned long long* acc_w,
                int32_t* acc_y) {
  __shared__ unsigned long long s_w[kTS / 32];
  __shared__ int s_lo[kTS / 32], s_hi[kTS / 32];
  const WorkTile wt = tiles[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long w = 0ull;
  int lo = INT_MAX, hi = INT_MIN;
  if ((int)threadIdx.x < wt.rows) {
    const int64_t e = wt.row0 + threadIdx.x;
    w = pr.w ? pr.w[e] : 1u;
    if (w) lo = hi = f2ord(pr.y[e]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    w += __shfl_xor_sync(0xffffffffu, w, off);
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
  }
  if (lane == 0) {
    s_w[warp] = w;
    s_lo[warp] = lo;
    s_hi[warp] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kTS / 32; ++i) {
      w += s_w[i];
      lo = min(lo, s_lo[i]);
      hi = max(hi, s_hi[i]);
    }
    atomicAdd(&acc_w[wt.node], w);
    if (lo != INT_MAX) {
      atomicMin(&acc_y[2 * wt.node], lo);
      atomicMax(&acc_y[2 * wt.node + 1], hi);
    }
  }
}

// One CTA per tile: the node's centre and scales (every CTA of the node
// derives the same values), then the fixed-point moments of the tile's rows.
__global__ void __launch_bounds__(kTS)
    k_mse_moments(Problem pr, const WorkTile* __restrict__ tiles,
                  const unsigned long long* __restrict__ acc_w, const int32_t* __restrict__ acc_y,
                  long long* m1, long long* m2, double* mscale) {
  const WorkTile wt = tiles[blockIdx.x];
  const int a = wt.node;
  const double W = (double)acc_w[a];
  float c = 0.0f;
  double D = 0.0;
  if (acc_y[2 * a] != INT_MAX) {
    const double ylo = ord2f(acc_y[2 * a]), yhi = ord2f(acc_y[2 * a + 1]);
    c = (float)(0.5 * (ylo + yhi));
    // rounding is monotone: every |y - c| below is at most D
    D = fmax(yhi - (double)c, (double)c - ylo);
  }
  int s = 0, t = 0;
  if (W > 0.0 && D > 0.0) {
    int e1, e2;
    frexp(W * D * (1.0 + 0x1p-40), &e1);      // W D < 2^e1
    frexp(W * D * D * (1.0 + 0x1p-40), &e2);  // W D^2 < 2^e2
    s = 61 - e1;
    t = e2 + 2 * s - 61;
  }
  if (threadIdx.x == 0) {  // identical from every tile of the node
    mscale[2 * a] = ldexp(1.0, -s);
    mscale[2 * a + 1] = ldexp(1.0, t - 2 * s);
  }
  if ((int)threadIdx.x >= wt.rows) return;
  const int64_t e = wt.row0 + threadIdx.x;
  const double w = pr.w ? (double)pr.w[e] : 1.0;
  const double v = (double)pr.y[e] - (double)c;
  m1[e] = llrint(w * v * ldexp(1.0, s));
  m2[e] = llrint(w * v * v * ldexp(1.0, 2 * s - t));
}

}  // namespace

// ---- launchers ---------------------------------------------------------------------

cudaError_t launch_mse_moments(const Problem& pr, const WorkTile* tiles, int n_tiles, int A,
                               unsigned long long* acc_w, int32_t* acc_y, long long* m1,
                               long long* m2, double* mscale, cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  k_mse_init<<<(A + 255) / 256, 256, 0, st>>>(A, acc_w, acc_y);
  if (n_tiles > 0) {
    k_mse_range<<<n_tiles, kTS, 0, st>>>(pr, tiles, acc_w, acc_y);
    k_mse_moments<<<n_tiles, kTS, 0, st>>>(pr, tiles, acc_w, acc_y, m1, m2, mscale);
  }
  return cudaGetLastError();
}

static size_t hist_smem_bytes(const Problem& pr) {
  const size_t hist =
      (hist_copy_bytes(pr.crit, pr.B, pr.K) * hist_copies(pr.crit) + 127) & ~(size_t)127;
  return hist + sort_bytes(pr.crit, pr.B) + kStages * stage_bytes(pr.crit, pr.w != nullptr);
}

cudaError_t prepare_eval_kernels(const Problem& pr) {
  cudaError_t e = cudaSuccess;
  for (const void* f : {(const void*)k_project<8>, (const void*)k_project<16>,
                        (const void*)k_project<24>, (const void*)k_project<32>,
                        (const void*)k_project<48>})
    if ((e = allow_smem((const void*)f, (int)kProjSmem)))
      return e;
  for (const void* f : {(const void*)k_project_tma<8>, (const void*)k_project_tma<16>,
                        (const void*)k_project_tma<24>, (const void*)k_project_tma<32>,
                        (const void*)k_project_tma<48>})
    if ((e = allow_smem((const void*)f, (int)kProjTmaSmem)))
      return e;
  for (const void* f : {(const void*)k_node_search<SLM_GINI>,
                        (const void*)k_node_search<SLM_ENTROPY>})
    if ((e = allow_smem((const void*)f, (int)kNodeSearchMaxSmem)))
      return e;
  for (const void* f : {(const void*)k_hist_warp<SLM_GINI>, (const void*)k_hist_warp<SLM_ENTROPY>})
    if ((e = allow_smem((const void*)f, (int)kHistWarpMaxSmem)))
      return e;
  if ((e = allow_smem((const void*)k_hist_scan, (int)hist_smem_bytes(pr))))
    return e;
  return allow_cluster((const void*)k_hist_scan);
}

cudaError_t launch_swarm_init(const Problem& pr, const Swarm& sw,
                              const NodeDesc* nodes, int A, SwarmCoef co,
                              cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  k_swarm_init<<<A, kThreads, 0, st>>>(pr, sw, nodes, co);
  return cudaGetLastError();
}

cudaError_t set_first_wait_polls(int polls) {
  const int v = polls < 0 ? kWaitPolls : polls;
  return cudaMemcpyToSymbol(d_first_wait_polls, &v, sizeof(v));
}

static std::mutex g_xlogx_mu;
static std::vector<const double*> g_xlogx_tabs;  // per device, under g_xlogx_mu

cudaError_t ensure_xlogx_table(int device) {
  static std::vector<char> done;
  std::lock_guard<std::mutex> lock(g_xlogx_mu);
  if ((int)done.size() <= device) done.resize(device + 1, 0);
  if (done[device]) return cudaSuccess;
  double* tab = nullptr;
  cudaError_t e = cudaMalloc(&tab, sizeof(double) * kXlogxTab);  // kept for the process
  if (e) return e;
  cudaStream_t st = nullptr;
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) return e;
  k_xlogx_table<<<(kXlogxTab + 255) / 256, 256, 0, st>>>(tab, kXlogxTab);
  if (!(e = cudaGetLastError())) e = cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (!e) e = cudaMemcpyToSymbol(d_xlogx_tab, &tab, sizeof(tab));
  if (!e) {
    done[device] = 1;
    if ((int)g_xlogx_tabs.size() <= device) g_xlogx_tabs.resize(device + 1, nullptr);
    g_xlogx_tabs[device] = tab;
  }
  return e;
}

const double* xlogx_table(int device) {
  std::lock_guard<std::mutex> lock(g_xlogx_mu);
  return device >= 0 && device < (int)g_xlogx_tabs.size() ? g_xlogx_tabs[device] : nullptr;
}

bool project_group_ok(const Problem& pr, int pg) {
  return (pg == 8 || pg == 16 || pg == 24 || pg == 32 || pg == 48) && pr.Pp % pg == 0;
}

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null if the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  });
  return fn;
}

// A row-major [rows, d] float tensor as boxes of box_rows rows x kKC
// features with 128-byte swizzle (d % 4 == 0, base 16-byte aligned). The
// last few encodings are kept per host thread: a search launches the same
// maps every iteration.
bool encode_rows(CUtensorMap* m, const float* base, uint64_t rows, int d, uint32_t box_rows) {
  struct Entry {
    const float* base;
    uint64_t rows;
    int d;
    uint32_t box_rows;
    bool ok;
    CUtensorMap map;
  };
  constexpr int kKeep = 8;
  thread_local Entry kept[kKeep];
  thread_local int n_kept = 0, next = 0;
  for (int i = 0; i < n_kept; ++i) {
    const Entry& e = kept[i];
    if (e.base == base && e.rows == rows && e.d == d && e.box_rows == box_rows) {
      if (e.ok) *m = e.map;
      return e.ok;
    }
  }
  Entry& e = kept[next];
  next = (next + 1) % kKeep;
  if (n_kept < kKeep) ++n_kept;
  e.base = base;
  e.rows = rows;
  e.d = d;
  e.box_rows = box_rows;
  e.ok = false;
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || rows == 0 || (d & 3) || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)d * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kKC, box_rows};
  const cuuint32_t es[2] = {1, 1};
  e.ok = enc(&e.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
             strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
  if (e.ok) *m = e.map;
  return e.ok;
}

}  // namespace

cudaError_t launch_project(const Problem& pr_in, const Swarm& sw, const WorkTile* tiles,
                           int n_tiles, int grid_cap, cudaStream_t st, int pg, bool gather,
                           int A) {
  Problem pr = pr_in;
  if (!gather || !pr.Xg) pr.gidx = nullptr;
  if (pg > 0) {
    if (!project_group_ok(pr, pg)) return cudaErrorInvalidValue;
    pr.G = pr.Pp / pg;
  }
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
  // contiguous rows: tensor-map tile copies (A > 0 names the batch's nodes,
  // which bound the positions' tensor)
  CUtensorMap tx, ta;
  const int PG = pr.Pp / pr.G;
  if (A > 0 && !pr.gidx && encode_rows(&tx, pr.X, (uint64_t)pr.E, pr.d, kTS) &&
      encode_rows(&ta, sw.pos, (uint64_t)A * pr.Pp, pr.d, (uint32_t)PG)) {
    cfg.dynamicSmemBytes = kProjTmaSmem;
    switch (PG) {
      case 8: return cudaLaunchKernelEx(&cfg, k_project_tma<8>, tx, ta, pr, sw, tiles, n_units);
      case 16: return cudaLaunchKernelEx(&cfg, k_project_tma<16>, tx, ta, pr, sw, tiles, n_units);
      case 24: return cudaLaunchKernelEx(&cfg, k_project_tma<24>, tx, ta, pr, sw, tiles, n_units);
      case 32: return cudaLaunchKernelEx(&cfg, k_project_tma<32>, tx, ta, pr, sw, tiles, n_units);
      case 48: return cudaLaunchKernelEx(&cfg, k_project_tma<48>, tx, ta, pr, sw, tiles, n_units);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (pr.Pp / pr.G) {
    case 8: return cudaLaunchKernelEx(&cfg, k_project<8>, pr, sw, tiles, n_units);
    case 16: return cudaLaunchKernelEx(&cfg, k_project<16>, pr, sw, tiles, n_units);
    case 24: return cudaLaunchKernelEx(&cfg, k_project<24>, pr, sw, tiles, n_units);
    case 32: return cudaLaunchKernelEx(&cfg, k_project<32>, pr, sw, tiles, n_units);
    case 48: return cudaLaunchKernelEx(&cfg, k_project<48>, pr, sw, tiles, n_units);
    default: return cudaErrorInvalidValue;
  }
}

int hist_split(const Problem& pr, int A, int64_t max_len, int n_sm, int max_cluster) {
  // clusters of S CTAs per (node, particle): as many as keep the whole grid
  // resident in one wave, with slices of at least one staged piece
  int per_sm = 1;
  if (occupancy(&per_sm, (const void*)k_hist_scan, kThreads, hist_smem_bytes(pr)) !=
      cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int64_t resident = (int64_t)(per_sm > 0 ? per_sm : 1) * n_sm;
  int S = 1;
  while (2 * S <= max_cluster && (int64_t)A * pr.P * (2 * S) <= resident &&
         max_len / (2 * S) >= piece_of(pr.crit, pr.w != nullptr))
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
                             int A, int S, int32_t* bins_out, int t, int do_update,
                             cudaStream_t st, const int32_t* list) {
  if (A <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(A * S), (unsigned)pr.P, 1);
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
  return cudaLaunchKernelEx(&cfg, k_hist_scan, pr, sw, nodes, list, bins_out, t, do_update);
}

size_t node_search_smem(const Problem& pr, int n, int S) {
  if (pr.d % 4 || S < 1) return SIZE_MAX;  // 16-byte row chunks
  const size_t slots = node_search_slots(pr.P, S);
  const size_t floats = (size_t)n * pr.d + (size_t)8 * n + 3 * slots * pr.d + pr.d;
  const size_t words = (size_t)8 * pr.B * pr.K + (size_t)n * (pr.w ? 2 : 1);
  return (floats * 4 + sizeof(EvalRes) * (2 * slots + pr.P) + words * 4 + 15) & ~(size_t)15;
}

cudaError_t launch_node_search(const Problem& pr, const Swarm& sw, const NodeDesc* nodes,
                               const int32_t* list, int n_nodes, int A, int S, size_t smem,
                               SwarmCoef co, cudaStream_t st) {
  if (n_nodes <= 0) return cudaSuccess;
  if (pr.crit == SLM_MSE || smem > kNodeSearchMaxSmem || S < 1 || S > 8)
    return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)S, (unsigned)n_nodes, 1);
  cfg.blockDim = dim3(kNodeThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
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
  if (pr.crit == SLM_GINI)
    return cudaLaunchKernelEx(&cfg, k_node_search<SLM_GINI>, pr, sw, nodes, list, A, co);
  return cudaLaunchKernelEx(&cfg, k_node_search<SLM_ENTROPY>, pr, sw, nodes, list, A, co);
}

size_t hist_warp_smem_bytes(const Problem& pr) {
  return sizeof(uint32_t) * (size_t)(kThreads / 32) * pr.B * pr.K;
}

bool hist_warp_ok(const Problem& pr) {
  return pr.crit != SLM_MSE && hist_warp_smem_bytes(pr) <= kHistWarpMaxSmem;
}

cudaError_t launch_hist_warp(const Problem& pr, const Swarm& sw, const NodeDesc* nodes,
                             const int32_t* list, int n_nodes, int t, int do_update,
                             cudaStream_t st) {
  const int64_t pairs = (int64_t)n_nodes * pr.P;
  if (pairs <= 0) return cudaSuccess;
  if (!hist_warp_ok(pr)) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((pairs + kThreads / 32 - 1) / (kThreads / 32)), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = hist_warp_smem_bytes(pr);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (pr.crit == SLM_GINI)
    return cudaLaunchKernelEx(&cfg, k_hist_warp<SLM_GINI>, pr, sw, nodes, list, (int)pairs, t,
                              do_update);
  return cudaLaunchKernelEx(&cfg, k_hist_warp<SLM_ENTROPY>, pr, sw, nodes, list, (int)pairs, t,
                            do_update);
}

cudaError_t launch_apso(const Problem& pr, const Swarm& sw, const NodeDesc* nodes, int A,
                        int t, SwarmCoef co, cudaStream_t st, const int32_t* list, int n_list) {
  const int n_nodes = list ? n_list : A;
  if (n_nodes <= 0 || !sw.apso) return cudaSuccess;
  const int R = apso_rows(pr.P, pr.d);
  if (R == 0) return cudaErrorInvalidValue;
  const size_t smem = apso_smem(pr.P, pr.d, R);
  cudaError_t e = allow_smem((const void*)k_apso, (int)smem);
  if (e) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)n_nodes, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_apso, pr, sw, nodes, t, co, list, A, R);
}

cudaError_t launch_move(const Problem& pr, const Swarm& sw, const NodeDesc* nodes, int A,
                        int t, SwarmCoef co, cudaStream_t st, const int32_t* list, int n_list) {
  const int n_nodes = list ? n_list : A;
  if (n_nodes <= 0) return cudaSuccess;
  const int items = pr.P * ((pr.d + 3) / 4);
  const int per_node = t >= sw.T ? 1 : (items + 127) / 128;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)n_nodes, (unsigned)per_node, 1);
  cfg.blockDim = dim3(128, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_move, pr, sw, nodes, t, co, list, A);
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
