// One iteration's projection of the FP32 swarm search with the swarm move
// folded in (Sec. III-A, Eq. pso-1 and Algorithm 1; Sec. II-A, Eq. 1).
//
// A search iteration t is two launches: k_step (gbest step of evaluation t-1,
// the move to x_t, z = X_node . x_t and the per-particle ranges) and a
// histogram kernel (bins, threshold scan, pbest step, and the gB-independent
// terms of the next move). k_step's unit is one tile of rows of one node with
// ALL of the node's particles, so every row tile is read from L2 once per
// iteration; the node's positions live in shared memory for the whole unit.
//
// The move needs gB, which needs every particle's score, so it cannot run in
// the histogram kernel that produces those scores. Every CTA that projects a
// node therefore takes the node's gbest step itself (a warp argmin over P
// scores) and forms the node's new positions from the terms the histogram
// kernel left: x' = x + (ic + s2 (gB - x)), three operations per element. The
// CTA holding the node's first row tile writes x' and v' back (into the
// other of two position buffers, so the other CTAs still read x) together
// with the gbest records, exactly as k_move would.
//
// Each CTA of the persistent grid takes a contiguous run of units; it forms a
// node's positions once for all its consecutive units of that node. The row
// tiles stream through a ring of shared-memory stages (the copies of the next
// NS - 1 feature chunks in flight, one barrier per chunk), and a finished
// unit's z leaves through per-warp staging rows, so that each store writes
// whole 128-byte rows of a particle.
//
// Thread tile: 4 rows (sg + 8i) x PJ particles (pg + 4j) per thread; a warp
// covers 32 rows x 4 PJ particles; the CTA's 8 warps are RB = 8 / PB row
// blocks x PB particle blocks, so a unit is 32 RB rows x 4 PJ PB = Pp
// particles. Every z is the sequential fused multiply-add over the features
// of k_project (bit-identical results).
#include <cuda_runtime.h>
#include <float.h>
#include <limits.h>

#include "device_util.cuh"
#include "slm_internal.cuh"

namespace slm {
namespace {

constexpr int kStepMaxPosBytes = 96 * 1024;  // the node's positions in shared memory
// Floats per particle of a warp's z staging rows: 32 rows and 8 of padding,
// so that the four particles a warp stages fall on distinct banks.
constexpr int kZS = 40;

// Positions in shared memory, chunk-major: feature j of particle p at
// (j / kKC) * Pp * kXS + p * kXS + j % kKC, so that the particles a thread
// reads sit at compile-time offsets and the four particles a warp reads at
// one feature fall on distinct banks (rows kXS = 36 floats apart). Features
// past d and particles past P stay zero.
__host__ __device__ inline size_t step_pos_floats(int Pp, int d) {
  return (size_t)((d + kKC - 1) / kKC) * Pp * kXS;
}

// Row-tile stages in the ring: the copies of the next NS - 1 steps are in
// flight while a step computes (fewer for the larger row tiles, so that two
// CTAs still fit on an SM).
__host__ __device__ constexpr int step_stages(int RT) { return RT <= 64 ? 4 : RT <= 128 ? 3 : 2; }

template <int PJ, int PB>
__global__ void __launch_bounds__(kThreads, 2)
    k_step(Problem pr, Swarm sw, const float* __restrict__ pos_prev,
           const NodeDesc* __restrict__ nodes, int A, const WorkTile* __restrict__ tiles,
           int n_units, int t) {
  constexpr int RB = 8 / PB;   // 32-row blocks of a unit
  constexpr int RT = 32 * RB;  // rows of a unit
  constexpr int PPB = 4 * PJ;  // particles of a particle block
  constexpr int PU = PPB * PB;  // particles of a unit (a slice of the swarm, or all of it)
  constexpr int NS = step_stages(RT);
  static_assert(PJ % 2 == 0 && RB * PB == 8 && NS >= 2, "tile shape");
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_lo[64], s_hi[64];  // ordered-int range of each particle
  __shared__ int s_best;
  const int d = pr.d, Pp = pr.Pp, P = pr.P;
  float* xs = sm;                                   // [NS][RT][kXS] row-tile stages
  float* ps = sm + NS * RT * kXS;                   // the node's positions, chunk-major
  float* gs = ps + step_pos_floats(Pp, d);          // the node's gB (d floats, padded to 4)
  float* zst = gs + ((d + 3) & ~3);                 // [8 warps][4][kZS] z staging rows
  pdl_trigger();
  const int nk = (d + kKC - 1) / kKC;
  const int cstride = Pp * kXS;   // floats per feature chunk of the positions
  const bool vec = (d & 3) == 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sg = lane & 7, pg = lane >> 3;
  const int rb = warp % RB, pbk = warp / RB;
  // a contiguous run of units per CTA (the tiles are in node order), so that
  // consecutive units of a CTA mostly share a node and its moved positions
  const int u0 = (int)(((int64_t)blockIdx.x * n_units) / gridDim.x);
  const int my_units = (int)(((int64_t)(blockIdx.x + 1) * n_units) / gridDim.x) - u0;
  const int n_st = my_units * nk;

  // rows of step s (unit s / nk, feature chunk s % nk) into its ring stage;
  // rows past the tile and features past d arrive as zeros. One commit group
  // per step, empty past the last.
  auto stage = [&](int s) {
    if (s < n_st) {
      float* xb = xs + (s % NS) * (RT * kXS);
      const int ui = s / nk, c = s - ui * nk;
      const WorkTile wt = tiles[u0 + ui];
      const int k0 = c * kKC, kc = min(kKC, d - k0);
      if (vec) {
        for (int q = threadIdx.x; q < RT * (kKC / 4); q += kThreads) {
          const int r = q >> 3, cc = (q & 7) * 4;
          const bool ok = r < wt.rows && cc < kc;
          const float* src = ok ? row_of(pr, wt.row0 + r) + k0 + cc : pr.X;
          cp_async16(xb + r * kXS + cc, src, ok ? 16 : 0);
        }
      } else {
        for (int q = threadIdx.x; q < RT * kKC; q += kThreads) {
          const int r = q >> 5, cc = q & 31;
          const bool ok = r < wt.rows && cc < kc;
          const float* src = ok ? row_of(pr, wt.row0 + r) + k0 + cc : pr.X;
          cp_async4(xb + r * kXS + cc, src, ok ? 4 : 0);
        }
      }
    }
    cp_async_commit();
  };

  if (threadIdx.x < 64) {
    s_lo[threadIdx.x] = INT_MAX;
    s_hi[threadIdx.x] = INT_MIN;
  }
  // Within a search the rows and tiles are written before the first
  // iteration's launch, so iterations t > 0 start fetching them before the
  // previous kernel's results are visible.
  if (t > 0)
    for (int s = 0; s < NS - 1; ++s) stage(s);
  // padding features and particles of the positions stay zero
  for (int i = threadIdx.x; i < nk * cstride; i += kThreads) ps[i] = 0.0f;
  pdl_wait();
  if (t == 0)
    for (int s = 0; s < NS - 1; ++s) stage(s);

  // The positions of node a for iteration t in ps (and, from the CTA that
  // holds the node's first row tile, in sw.pos / sw.vel with the gbest
  // records of evaluation t - 1).
  // desig: this CTA holds the first row tile of its slice (particles pg0 ..
  // pg0 + PU - 1) of node a; the slice's positions go back to memory from
  // there, and the node's gbest records from slice 0's
  auto node_positions = [&](int a, int pg0, bool desig) {
    const int64_t nb = (int64_t)a * Pp * d;
    const bool desig0 = desig && pg0 == 0;
    const int p_lo = min(pg0, P), p_hi = min(P, pg0 + PU);  // the slice's particles
    if (t == 0 || sw.node_step) {  // the histogram kernel moved the swarm
      for (int e = threadIdx.x; e < P * d; e += kThreads) {
        const int p = e / d, j = e - p * d;
        ps[(j / kKC) * cstride + p * kXS + j % kKC] = pos_prev[nb + e];
      }
      __syncthreads();
      return;
    }
    // Positions of t - 1 go by asynchronous copies straight into ps (moved
    // there in place) and the recorded gB into gs; the move terms to
    // registers; all before the gbest step. After a gbest change gB is the
    // new best particle's position of t - 1 (it beat every pbest, so its own
    // pbest became that position), which ps then holds: the move needs
    // nothing more from global memory.
    const int d4 = d >> 2, items = vec ? P * d4 : 0;
    // the slice's elements (the positions of every particle are copied: gB
    // may be any particle's)
    const int e_lo = vec ? p_lo * d4 : 0, e_hi = vec ? p_hi * d4 : 0;
    if (vec) {
      for (int e = threadIdx.x; e < items; e += kThreads) {
        const int p = e / d4, j = 4 * (e - p * d4);
        cp_async16(ps + (j / kKC) * cstride + p * kXS + j % kKC, pos_prev + nb + 4 * (int64_t)e,
                   16);
      }
      for (int q = threadIdx.x; q < d4; q += kThreads)
        cp_async16(gs + 4 * q, sw.gbest + (int64_t)a * d + 4 * q, 16);
      cp_async_commit();
    }
    // the move terms: every element of the thread in flight at once when
    // they fit kPre float4 per thread, else two at a time
    constexpr int kPre = 4;
    const bool pre = e_hi - e_lo <= kPre * kThreads;
    float4 ia[kPre], sa[kPre];
    auto load_terms = [&](int e0, int n) {
#pragma unroll
      for (int u = 0; u < kPre; ++u) {
        const int e = e0 + u * kThreads;
        if (u < n && e < e_hi) {
          const int64_t o = nb + 4 * (int64_t)e;  // element (p, 4q) of the node's rows
          ia[u] = __ldcg(reinterpret_cast<const float4*>(sw.ic + o));
          sa[u] = __ldcg(reinterpret_cast<const float4*>(sw.s2 + o));
        }
      }
    };
    load_terms(e_lo + threadIdx.x, pre ? kPre : 2);
    // gbest step of evaluation t - 1 (k_move's rule and double buffering),
    // its inputs loaded together: the node's scores (two per lane), the
    // improvement flag and the recorded gbest score
    if (warp == 0) {
      const EvalRes* cur = sw.cur + (int64_t)a * Pp;
      const EvalRes e0 = lane < P ? cur[lane] : invalid_res();
      const EvalRes e1 = lane + 32 < P ? cur[lane + 32] : invalid_res();
      // the argmin only when a particle beat gB in evaluation t - 1 (every
      // particle is a candidate at evaluation 0)
      const bool any = t == 1 || !sw.imp || __ldcg(sw.imp + (int64_t)((t - 1) & 1) * A + a) != 0;
      const EvalRes gold = sw.gb[(int64_t)(t & 1) * A + a];
      EvalRes be = gold;
      int bi = -1;
      if (any) {
        int ci = -1;
        EvalRes ce = invalid_res();
        if (lane < P) gbest_consider(pr, gold, t - 1, lane, e0, &ci, &ce);
        if (lane + 32 < P) gbest_consider(pr, gold, t - 1, lane + 32, e1, &ci, &ce);
        bi = gbest_select(pr, ci, ce, &be);
      }
      if (lane == 0) {
        s_best = bi;
        if (desig0 && sw.imp) sw.imp[(int64_t)(t & 1) * A + a] = 0;  // evaluation t's flag
        if (desig0) {
          const EvalRes g = bi >= 0 ? be : gold;
          sw.gb[(int64_t)((t - 1) & 1) * A + a] = g;
          if (bi >= 0) {
            sw.gpart[a] = bi;
            sw.giter[a] = t - 1;
          }
          if (sw.trace)
            sw.trace[(int64_t)a * (sw.T + 1) + (t - 1)] =
                g.valid ? g.loss : __longlong_as_double(0x7ff0000000000000LL);
        }
      }
    }
    if (vec) cp_async_wait<0>();
    __syncthreads();
    const int bi = s_best;
    if (vec) {
      // gB into gs before any position is overwritten
      if (bi >= 0)
        for (int j = threadIdx.x; j < d; j += kThreads)
          gs[j] = ps[(j / kKC) * cstride + bi * kXS + j % kKC];
      __syncthreads();
      if (desig0 && bi >= 0)
        for (int j = threadIdx.x; j < d; j += kThreads) sw.gbest[(int64_t)a * d + j] = gs[j];
      // x' = x + (ic + s2 (gB - x)), v' = ic + s2 (gB - x), one rounding each
      auto move4 = [&](int e, const float4& ic, const float4& s2) {
        const int p = e / d4, j = 4 * (e - p * d4);
        float* xp = ps + (j / kKC) * cstride + p * kXS + j % kKC;
        const float4 x = *reinterpret_cast<const float4*>(xp);
        const float4 g = *reinterpret_cast<const float4*>(gs + j);
        float4 vn, xn;
        vn.x = __fadd_rn(ic.x, __fmul_rn(s2.x, __fsub_rn(g.x, x.x)));
        vn.y = __fadd_rn(ic.y, __fmul_rn(s2.y, __fsub_rn(g.y, x.y)));
        vn.z = __fadd_rn(ic.z, __fmul_rn(s2.z, __fsub_rn(g.z, x.z)));
        vn.w = __fadd_rn(ic.w, __fmul_rn(s2.w, __fsub_rn(g.w, x.w)));
        xn.x = __fadd_rn(x.x, vn.x);
        xn.y = __fadd_rn(x.y, vn.y);
        xn.z = __fadd_rn(x.z, vn.z);
        xn.w = __fadd_rn(x.w, vn.w);
        if (desig) {
          const int64_t o = nb + 4 * (int64_t)e;
          *reinterpret_cast<float4*>(sw.pos + o) = xn;
          *reinterpret_cast<float4*>(sw.vel + o) = vn;
        }
        *reinterpret_cast<float4*>(xp) = xn;
      };
      if (pre) {
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
          const int e = e_lo + threadIdx.x + u * kThreads;
          if (e < e_hi) move4(e, ia[u], sa[u]);
        }
      } else {
        for (int e0 = e_lo + threadIdx.x; e0 < e_hi; e0 += 2 * kThreads) {
          if (e0 != e_lo + (int)threadIdx.x) load_terms(e0, 2);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int e = e0 + u * kThreads;
            if (e < e_hi) move4(e, ia[u], sa[u]);
          }
        }
      }
    } else {
      // a new best improved its pbest in evaluation t - 1: gB is that row
      const float* gsrc = bi >= 0 ? sw.pbest + nb + (int64_t)bi * d : sw.gbest + (int64_t)a * d;
      if (desig0 && bi >= 0)
        for (int j = threadIdx.x; j < d; j += kThreads) sw.gbest[(int64_t)a * d + j] = gsrc[j];
      for (int e = p_lo * d + (int)threadIdx.x; e < p_hi * d; e += kThreads) {
        const int p = e / d, j = e - p * d;
        const int64_t o = nb + e;
        const float x = pos_prev[o];
        const float vn = __fadd_rn(sw.ic[o], __fmul_rn(sw.s2[o], __fsub_rn(gsrc[j], x)));
        const float xn = __fadd_rn(x, vn);
        if (desig) {
          sw.pos[o] = xn;
          sw.vel[o] = vn;
        }
        ps[(j / kKC) * cstride + p * kXS + j % kKC] = xn;
      }
    }
    __syncthreads();
  };

  // the CTA's range of each particle of node a, into the node's ranges
  auto flush_ranges = [&](int a) {
    if ((int)threadIdx.x < P && s_lo[threadIdx.x] != INT_MAX) {
      int* zz = sw.zmm + ((int64_t)a * Pp + threadIdx.x) * 2;
      atomicMin(zz, s_lo[threadIdx.x]);
      atomicMax(zz + 1, s_hi[threadIdx.x]);
    }
    if (threadIdx.x < 64) {
      s_lo[threadIdx.x] = INT_MAX;
      s_hi[threadIdx.x] = INT_MIN;
    }
  };

  float acc[4][PJ];
  int cur_a = -1, cur_pg = -1;
  float* zw = zst + warp * (4 * kZS);  // this warp's staging rows
  const bool z16 = ((reinterpret_cast<uintptr_t>(sw.z) | (uintptr_t)pr.Ez * 4) & 15) == 0;

  for (int s = 0; s < n_st; ++s) {
    const int ui = s / nk, c = s - ui * nk;
    const WorkTile wt = tiles[u0 + ui];
    cp_async_wait<NS - 2>();
    // step s's rows are in place, and every warp is done with step s - 1
    // (its stage, the positions of its node, its ranges)
    __syncthreads();
    if (c == 0) {  // a unit starts (no sum is live through the move)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < PJ; ++j) acc[i][j] = 0.0f;
      if (wt.node != cur_a || wt.pad != cur_pg) {
        if (cur_a >= 0) flush_ranges(cur_a);
        cur_a = wt.node;
        cur_pg = wt.pad;
        node_positions(cur_a, cur_pg, wt.row0 == nodes[cur_a].seg_start);
      }
    }
    stage(s + NS - 1);  // into the stage step s - 1 read
    const float* xr = xs + (s % NS) * (RT * kXS) + (rb * 32 + sg) * kXS;
    const float* ar = ps + c * cstride + (cur_pg + pbk * PPB + pg) * kXS;
    // features 4 ch .. 4 ch + 3 of the chunk: feature-outer within each pair
    // of particles, so every accumulator takes the features in increasing order
    auto fma4 = [&](int ch) {
      float4 xv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        xv[i] = *reinterpret_cast<const float4*>(xr + i * 8 * kXS + 4 * ch);
#pragma unroll
      for (int j = 0; j < PJ; j += 2) {
        const float4 a0 = *reinterpret_cast<const float4*>(ar + j * 4 * kXS + 4 * ch);
        const float4 a1 = *reinterpret_cast<const float4*>(ar + (j + 1) * 4 * kXS + 4 * ch);
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
    };
    const int kc4 = (min(kKC, d - c * kKC) + 3) >> 2;  // 16-byte chunks of features
    if (kc4 == kKC / 4) {
#pragma unroll(PJ <= 4 ? 2 : 1)
      for (int ch = 0; ch < kKC / 4; ++ch) fma4(ch);
    } else {
#pragma unroll 1
      for (int ch = 0; ch < kc4; ++ch) fma4(ch);
    }
    if (c == nk - 1) {
      // unit complete: the ranges into the CTA's; z out through the warp's
      // staging rows, so that every store writes whole rows of a particle
      // (four 128-byte rows per 16-byte store when aligned, else one per
      // 4-byte store) instead of 32-byte pieces of four rows
      const int rw = wt.rows - rb * 32;  // rows of the warp's block in the tile
      const int64_t zrow = wt.row0 + rb * 32;
      const bool v16 = z16 && rw >= 32 && (zrow & 3) == 0;
#pragma unroll
      for (int j = 0; j < PJ; ++j) {
        const int pb0 = cur_pg + pbk * PPB + 4 * j;  // the warp's particles pb0 .. pb0 + 3
        const int p = pb0 + pg;
        float lo = FLT_MAX, hi = -FLT_MAX;
        bool any = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (sg + 8 * i < rw) {
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
        if (sg == 0 && olo != INT_MAX && p < P) {
          atomicMin(&s_lo[p], olo);
          atomicMax(&s_hi[p], ohi);
        }
        __syncwarp();  // the previous particles' staging rows are read
#pragma unroll
        for (int i = 0; i < 4; ++i) zw[pg * kZS + sg + 8 * i] = acc[i][j];
        __syncwarp();
        if (v16) {
          const int q = lane >> 3, r4 = 4 * (lane & 7);
          const float4 v = *reinterpret_cast<const float4*>(zw + q * kZS + r4);
          if (pb0 + q < P) *reinterpret_cast<float4*>(sw.z + (int64_t)(pb0 + q) * pr.Ez + zrow + r4) = v;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (lane < rw && pb0 + q < P) sw.z[(int64_t)(pb0 + q) * pr.Ez + zrow + lane] = zw[q * kZS + lane];
        }
      }
    }
  }
  __syncthreads();  // every warp's ranges are in
  if (cur_a >= 0) flush_ranges(cur_a);
}

// Tile shapes of a padded swarm, largest row tile first: (PJ, PB), rows per
// unit 32 (8 / PB), particles per unit 4 PJ PB. Shapes 0-2 take every
// particle in a unit; shapes 3-5 take half of them (two slices of a swarm of
// 32 or 64), so a short node is spread over twice the CTAs with half the
// move and projection each. The smaller tiles spread a short node further.
constexpr int kStepShapes = 6;

bool step_shape(int Pp, int sh, int* PJ, int* PB) {
  static const int tab[4][3][2] = {
      {{4, 1}, {2, 2}, {0, 0}},   // 16 particles per unit
      {{8, 1}, {4, 2}, {2, 4}},   // 32
      {{6, 2}, {0, 0}, {0, 0}},   // 48
      {{8, 2}, {4, 4}, {2, 8}}};  // 64
  if (Pp % 16 || Pp < 16 || Pp > 64 || sh < 0 || sh >= kStepShapes) return false;
  const int pu = sh < 3 ? Pp : Pp / 2;  // particles per unit
  if (pu % 16) return false;
  const int* e = tab[pu / 16 - 1][sh % 3];
  *PJ = e[0];
  *PB = e[1];
  return e[0] > 0;
}

size_t step_smem(const Problem& pr, int sh) {
  int PJ = 0, PB = 0;
  if (!step_shape(pr.Pp, sh, &PJ, &PB)) return 0;
  const int RT = 32 * (8 / PB);
  return sizeof(float) * ((size_t)step_stages(RT) * RT * kXS + step_pos_floats(pr.Pp, pr.d) +
                          (size_t)((pr.d + 3) & ~3) + (size_t)8 * 4 * kZS);
}

template <class F>
cudaError_t step_dispatch(int Pp, int sh, F&& f) {
  int PJ = 0, PB = 0;
  if (!step_shape(Pp, sh, &PJ, &PB)) return cudaErrorInvalidValue;
  switch (PJ * 16 + PB) {
    case 4 * 16 + 1: return f(k_step<4, 1>);
    case 2 * 16 + 2: return f(k_step<2, 2>);
    case 8 * 16 + 1: return f(k_step<8, 1>);
    case 4 * 16 + 2: return f(k_step<4, 2>);
    case 2 * 16 + 4: return f(k_step<2, 4>);
    case 6 * 16 + 2: return f(k_step<6, 2>);
    case 8 * 16 + 2: return f(k_step<8, 2>);
    case 4 * 16 + 4: return f(k_step<4, 4>);
    case 2 * 16 + 8: return f(k_step<2, 8>);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool step_ok(const Problem& pr) {
  int PJ = 0, PB = 0;
  return step_shape(pr.Pp, 0, &PJ, &PB) &&
         step_pos_floats(pr.Pp, pr.d) * sizeof(float) <= (size_t)kStepMaxPosBytes;
}

int step_rows(const Problem& pr, int sh) {
  int PJ = 0, PB = 0;
  return step_shape(pr.Pp, sh, &PJ, &PB) ? 32 * (8 / PB) : 0;
}

int step_slices(const Problem& pr, int sh) {
  int PJ = 0, PB = 0;
  return step_shape(pr.Pp, sh, &PJ, &PB) ? pr.Pp / (4 * PJ * PB) : 0;
}

cudaError_t prepare_step_kernels(const Problem& pr, int sh) {
  return step_dispatch(pr.Pp, sh, [&](auto fn) {
    return allow_smem((const void*)fn, (int)step_smem(pr, sh));
  });
}

int step_grid(const Problem& pr, int sh, int n_sm) {
  int per_sm = 0;
  const cudaError_t e = step_dispatch(pr.Pp, sh, [&](auto fn) {
    return occupancy(&per_sm, (const void*)fn, kThreads, step_smem(pr, sh));
  });
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * n_sm;
}

cudaError_t launch_step(const Problem& pr, const Swarm& sw, const float* pos_prev,
                        const NodeDesc* nodes, int A, const WorkTile* tiles, int n_tiles,
                        int grid, int sh, int t, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  if (!step_ok(pr) || grid <= 0) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_tiles < grid ? n_tiles : grid), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = step_smem(pr, sh);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return step_dispatch(pr.Pp, sh, [&](auto fn) {
    return cudaLaunchKernelEx(&cfg, fn, pr, sw, pos_prev, nodes, A, tiles, n_tiles, t);
  });
}

}  // namespace slm
