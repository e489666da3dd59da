// Reduced-precision scoring on the 5th-generation tensor cores, and the
// top-k re-scoring of SLM_PROJ_BF16_TOPK.
//
// Scoring pass (Sec. II-A, Eq. 1, with bfloat16 operands):
//   z[p][e] = sum_k bf16(X[e][k]) * bf16(x_p[k]),   FP32 accumulation,
// the dense (rows x d) . (d x P) product of a node. A CTA owns kMmaRows = 128
// rows of one node at a time. One thread issues tcgen05.mma (kind::f16, BF16
// A and B, FP32 accumulator in tensor memory, M = 128, N = P', K = 16 per
// instruction) on operands that 1D bulk copies stage in shared memory; the
// four warps read the accumulator back with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31 = rows of the tile), store z to the L2-resident z buffer and
// fold each particle's range. The level's rows are converted to bfloat16 once
// per level, directly into the operand layout, so a tile chunk is one
// contiguous copy; the positions are converted once per iteration.
//
// Then, per node, the k particles with the best such score (selected by the
// last histogram CTA of the node) are re-scored on the FP32 projection (the
// k_project / k_hist_scan path) and k_merge writes their scores over the
// reduced ones, takes every particle's pbest step and the gbest step among
// the re-scored particles (Algorithm 1).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <limits.h>

#include "device_util.cuh"
#include "slm_internal.cuh"

namespace slm {
namespace {

constexpr int kMmaKC = 128;       // features per staged chunk of a tile
constexpr int kMmaThreads = 128;  // four warps: the 128 TMEM lanes

// ---- tensor memory and tcgen05 -------------------------------------------------

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                   smem_addr(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// Shared-memory matrix descriptor, K-major and unswizzled: core matrices of
// 8 rows x 16 bytes (128 contiguous bytes); the two core matrices of one
// 16-element K step lie lbo bytes apart, consecutive 8-row groups sbo apart.
__device__ __forceinline__ uint64_t mma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // fixed field of the tcgen05 descriptor format
  return d;                // base offset 0, relative LBO, no swizzle
}
// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, no negation or sparsity, shape M x N.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// bar receives one arrival once every MMA this thread issued has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_addr(bar))
      : "memory");
}
// 16 consecutive 32-bit accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

// ---- operand layout ----------------------------------------------------------------

// One thread per 16 bytes of output, in output order: block b of R rows,
// 16-feature step ks, 8-row group rg, 8-feature half kc, row r8 of the group.
__global__ void k_to_mma_layout(const float* __restrict__ src, int64_t n_src_rows, int d, int dp,
                                int R, int64_t n_units, uint4* __restrict__ out) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n_units) return;
  const int64_t per_block = (int64_t)R * dp / 8;
  const int64_t b = u / per_block;
  const int rem = (int)(u - b * per_block);
  const int ks = rem / (2 * R), rem2 = rem - ks * 2 * R;
  const int rg = rem2 >> 4, kc = (rem2 >> 3) & 1, r8 = rem2 & 7;
  const int64_t row = b * R + rg * 8 + r8;
  const int k0 = ks * 16 + kc * 8;
  float v[8];
  if (row < n_src_rows && (d & 3) == 0 && k0 + 8 <= d) {
    const float4* s = reinterpret_cast<const float4*>(src + row * d + k0);
    const float4 p0 = s[0], p1 = s[1];
    v[0] = p0.x; v[1] = p0.y; v[2] = p0.z; v[3] = p0.w;
    v[4] = p1.x; v[5] = p1.y; v[6] = p1.z; v[7] = p1.w;
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c)
      v[c] = (row < n_src_rows && k0 + c < d) ? src[row * d + k0 + c] : 0.0f;
  }
  out[u] = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                      pack_bf16x2(v[6], v[7]));
}

// ---- projection ----------------------------------------------------------------------

__host__ __device__ inline uint32_t mma_stage_bytes(int dp) {
  return (uint32_t)kMmaRows * (uint32_t)(dp < kMmaKC ? dp : kMmaKC) * 2u;
}
__host__ __device__ inline uint32_t mma_tmem_cols(int Pp) {
  uint32_t c = 32;
  while (c < (uint32_t)Pp) c <<= 1;
  return c;
}

// Persistent over the tiles blockIdx.x, blockIdx.x + gridDim.x, ...; each
// tile is one or more kMmaKC-feature chunks ("items"). Thread 0 streams the
// items through two shared-memory stages (bulk copies, mbarrier full[s]),
// issues the MMAs of an item as soon as it lands and commits them to
// free[s] (stage reusable) and, after the tile's last chunk, to acc[u & 1]:
// the accumulator is double-buffered in tensor memory, so the MMAs of tile
// u+1 run while the four warps read tile u back. The positions of a node are
// staged once per node. Each warp keeps a running range per column in shared
// memory, folded into global memory once per node.
__global__ void __launch_bounds__(kMmaThreads)
    k_project_mma(Problem pr, Swarm sw, const WorkTile* __restrict__ tiles, int n_tiles,
                  const uint16_t* __restrict__ posb) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_full[2], bar_free[2], bar_acc[2], bar_b;
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  __shared__ int s_lo[kMmaThreads / 32][kMaxParticles], s_hi[kMmaThreads / 32][kMaxParticles];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int P = pr.P, Pp = pr.Pp, dp = pr.dp;
  const uint32_t stage = mma_stage_bytes(dp);
  unsigned char* As = smem;
  unsigned char* Bs = smem + 2 * stage;
  const uint32_t b_bytes = (uint32_t)Pp * (uint32_t)dp * 2u;
  const uint32_t cols = mma_tmem_cols(Pp);  // one accumulator; two are allocated
  const int nch = (dp + kMmaKC - 1) / kMmaKC;
  const uint32_t idesc = mma_idesc(kMmaRows, Pp);

  if (warp == 0) {
    tmem_alloc(&s_tmem, 2 * cols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar_full[i], 1);
      mbar_init(&bar_free[i], 1);
      mbar_init(&bar_acc[i], 1);
    }
    mbar_init(&bar_b, 1);
    mbar_init_fence();
    s_err = 0;
  }
  for (int p = lane; p < Pp; p += 32) {  // each warp its own running range
    s_lo[warp][p] = INT_MAX;
    s_hi[warp][p] = INT_MIN;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  pdl_trigger();
  pdl_wait();

  const int my_tiles =
      (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int n_items = my_tiles * nch;
  auto tile_of = [&](int ti) { return tiles[blockIdx.x + ti * gridDim.x]; };
  auto wait_bar = [&](uint64_t* bar, uint32_t parity) {
    if (!mbar_wait(bar, parity, kWaitPolls)) s_err = 1;
  };
  // thread 0: bulk copy of item i into stage i & 1
  auto issue = [&](int i) {
    const int ti = i / nch, c = i - ti * nch;
    const WorkTile wt = tile_of(ti);
    const int k0 = c * kMmaKC;
    const int kl = dp - k0 < kMmaKC ? dp - k0 : kMmaKC;
    const uint32_t bytes = (uint32_t)kMmaRows * (uint32_t)kl * 2u;
    const uint16_t* src = pr.Xb + ((int64_t)(wt.row0 / kMmaRows) * dp + k0) * kMmaRows;
    mbar_expect_tx(&bar_full[i & 1], bytes);
    bulk_g2s(As + (i & 1) * stage, src, bytes, &bar_full[i & 1]);
  };
  // thread 0: every MMA of tile ti into accumulator ti & 1
  int b_node = -1;
  uint32_t b_phase = 0;
  auto mma_tile = [&](int ti) {
    const WorkTile wt = tile_of(ti);
    if (wt.node != b_node) {
      // the MMAs of tile ti-1 read the staged positions: let them finish
      if (ti > 0) wait_bar(&bar_acc[(ti - 1) & 1], (uint32_t)(((ti - 1) >> 1) & 1));
      mbar_expect_tx(&bar_b, b_bytes);
      bulk_g2s(Bs, posb + (int64_t)wt.node * Pp * dp, b_bytes, &bar_b);
      wait_bar(&bar_b, b_phase);
      b_phase ^= 1u;
      b_node = wt.node;
    }
    const uint32_t d_tmem = tmem + (uint32_t)(ti & 1) * cols;
    for (int c = 0; c < nch; ++c) {
      const int i = ti * nch + c;
      if (i + 1 < n_items) {
        // stage (i+1)&1 last held item i-1: wait until its MMAs are done
        if (i >= 1) wait_bar(&bar_free[(i - 1) & 1], (uint32_t)(((i - 1) >> 1) & 1));
        issue(i + 1);
      }
      wait_bar(&bar_full[i & 1], (uint32_t)((i >> 1) & 1));
      tc_fence_after();
      const int k0 = c * kMmaKC;
      const int kl = dp - k0 < kMmaKC ? dp - k0 : kMmaKC;
      const uint32_t a0 = smem_addr(As + (i & 1) * stage);
      const uint32_t b0 = smem_addr(Bs);
      for (int j = 0; j < kl / 16; ++j) {
        const uint64_t ad = mma_desc(a0 + (uint32_t)j * (kMmaRows * 32), 128, 256);
        const uint64_t bd = mma_desc(b0 + (uint32_t)(k0 / 16 + j) * (uint32_t)(Pp * 32), 128, 256);
        mma_bf16(d_tmem, ad, bd, idesc, (c > 0 || j > 0) ? 1u : 0u);
      }
      mma_commit(&bar_free[i & 1]);
    }
    mma_commit(&bar_acc[ti & 1]);
  };

  if (tid == 0 && n_items > 0) {
    issue(0);
    mma_tile(0);
  }
  for (int ti = 0; ti < my_tiles; ++ti) {
    const WorkTile wt = tile_of(ti);
    // accumulator (ti+1)&1 was last read in iteration ti-1, before its barrier
    if (tid == 0 && ti + 1 < my_tiles) mma_tile(ti + 1);
    if (!mbar_wait(&bar_acc[ti & 1], (uint32_t)((ti >> 1) & 1), kWaitPolls)) s_err = 1;
    tc_fence_after();
    // epilogue: accumulator row r = 32 warp + lane holds z of every particle
    const int r = warp * 32 + lane;
    const bool rv = r < wt.rows;
    float* zrow = sw.z + wt.row0 + r;
    const uint32_t t_row = tmem + (uint32_t)(ti & 1) * cols + ((uint32_t)(warp * 32) << 16);
    for (int cb = 0; cb < Pp / 16; ++cb) {
      uint32_t v[16];
      tmem_ld16(t_row + (uint32_t)(cb * 16), v);
      int my_lo = INT_MAX, my_hi = INT_MIN;  // lane j < 16: column cb*16 + j
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int p = cb * 16 + j;
        const float z = __uint_as_float(v[j]);
        const int oz = f2ord(z);
        const int lo = __reduce_min_sync(0xffffffffu, rv ? oz : INT_MAX);
        const int hi = __reduce_max_sync(0xffffffffu, rv ? oz : INT_MIN);
        if (rv && p < P) zrow[(int64_t)p * pr.Ez] = z;
        my_lo = lane == j ? lo : my_lo;
        my_hi = lane == j ? hi : my_hi;
      }
      if (lane < 16) {
        const int p = cb * 16 + lane;
        s_lo[warp][p] = min(s_lo[warp][p], my_lo);
        s_hi[warp][p] = max(s_hi[warp][p], my_hi);
      }
    }
    tc_fence_before();
    const bool last_of_node = ti + 1 == my_tiles || tile_of(ti + 1).node != wt.node;
    if (last_of_node) {
      // fold the warps' ranges of this node and publish them
      __syncthreads();
      for (int p = tid; p < P; p += kMmaThreads) {
        int lo = INT_MAX, hi = INT_MIN;
#pragma unroll
        for (int w = 0; w < kMmaThreads / 32; ++w) {
          lo = min(lo, s_lo[w][p]);
          hi = max(hi, s_hi[w][p]);
          s_lo[w][p] = INT_MAX;
          s_hi[w][p] = INT_MIN;
        }
        if (lo != INT_MAX) {
          int* zz = sw.zmm + ((int64_t)wt.node * Pp + p) * 2;
          atomicMin(zz, lo);
          atomicMax(zz + 1, hi);
        }
      }
    }
    __syncthreads();  // accumulator ti & 1 and the range slots free again
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 2 * cols);
  if (tid == 0 && s_err && sw.err) atomicExch(sw.err, kErrMmaTimeout);
}

// ---- merge of the re-scored particles ----------------------------------------------------

// Grid (node, group of 8 particles): warp w of block y merges particle
// 8 y + w and takes its pbest step; block y = 0 also takes the node's gbest
// step among the re-scored particles, from their FP32 scores in cur2.
__global__ void __launch_bounds__(256)
    k_merge(Problem pr, Swarm sw, const EvalRes* __restrict__ cur2, int kp,
            const int32_t* __restrict__ inv, int t, int do_update) {
  __shared__ int s_best;
  pdl_trigger();
  pdl_wait();
  const int a = blockIdx.x, A = gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int Pp = pr.Pp, d = pr.d;
  const int p = blockIdx.y * 8 + warp;
  if (p < pr.P) {
    const int q = inv[(int64_t)a * Pp + p];
    const EvalRes e = q >= 0 ? cur2[(int64_t)a * kp + q] : sw.cur[(int64_t)a * Pp + p];
    if (q >= 0 && lane == 0) sw.cur[(int64_t)a * Pp + p] = e;
    if (do_update) pbest_step(pr, sw, a, p, t, e);
  }
  if (!do_update || blockIdx.y != 0) return;
  if (warp == 0) {
    // gbest step among the re-scored particles: the best strictly better
    // than the gbest of iteration t-1 (at t = 0 any), ties to the lower index
    const EvalRes gold = sw.gb[(int64_t)((t + 1) & 1) * A + a];
    int bi = -1;
    EvalRes be = invalid_res();
    for (int q = lane; q < sw.k; q += 32) {
      const int pq = sw.sel[(int64_t)a * sw.k + q];
      const EvalRes e = cur2[(int64_t)a * kp + q];
      if (!(t == 0 || better(e, gold, pr.crit))) continue;
      if (bi < 0 || better(e, be, pr.crit)) {
        bi = pq;
        be = e;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      const EvalRes o = shfl_res(be, lane ^ off);
      bool take;
      if (oi < 0)
        take = false;
      else if (bi < 0)
        take = true;
      else if (better(o, be, pr.crit))
        take = true;
      else if (better(be, o, pr.crit))
        take = false;
      else
        take = oi < bi;
      if (take) {
        bi = oi;
        be = o;
      }
    }
    if (lane == 0) {
      s_best = bi;
      const EvalRes g = bi >= 0 ? be : gold;
      sw.gb[(int64_t)(t & 1) * A + a] = g;
      if (bi >= 0) {
        sw.gpart[a] = bi;
        sw.giter[a] = t;
      }
      if (sw.trace)
        sw.trace[(int64_t)a * (sw.T + 1) + t] =
            g.valid ? g.loss : __longlong_as_double(0x7ff0000000000000LL);
    }
  }
  __syncthreads();
  const int best = s_best;
  if (best >= 0)  // gB <- the current position of the new best
    for (int j = threadIdx.x; j < d; j += blockDim.x)
      sw.gbest[(int64_t)a * d + j] = sw.pos[((int64_t)a * Pp + best) * d + j];
}

size_t mma_smem_bytes(const Problem& pr) {
  const size_t need = 2 * (size_t)mma_stage_bytes(pr.dp) + (size_t)pr.Pp * pr.dp * 2;
  // at most 512 / (2 cols) CTAs fit in an SM's tensor memory: ask for enough
  // shared memory that no more fit
  int dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
      cudaSuccess) {
    cudaGetLastError();
    per_sm = 233472;
  }
  const int max_ctas = (int)(512u / (2 * mma_tmem_cols(pr.Pp)));
  const size_t floor_bytes = ((size_t)per_sm / (size_t)(max_ctas + 1) + 128) & ~(size_t)127;
  return need > floor_bytes ? need : floor_bytes;
}

}  // namespace

// ---- launchers ---------------------------------------------------------------------

cudaError_t launch_to_mma_layout(const float* src, int64_t n_src_rows, int d, int dp, int R,
                                 int64_t n_blocks, uint16_t* out, cudaStream_t st) {
  const int64_t n_units = n_blocks * (int64_t)R * dp / 8;
  if (n_units <= 0) return cudaSuccess;
  k_to_mma_layout<<<(unsigned)((n_units + 255) / 256), 256, 0, st>>>(
      src, n_src_rows, d, dp, R, n_units, reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

cudaError_t prepare_mma_kernels(const Problem& pr) {
  cudaError_t e = cudaFuncSetAttribute(k_project_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)mma_smem_bytes(pr));
  if (e) return e;
  return cudaFuncSetAttribute(k_project_mma, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

int mma_grid_cap(const Problem& pr, int n_sm) {
  // resident CTAs per SM from the kernel's own limits: shared memory (static,
  // dynamic and the per-block reservation), tensor memory, 16 blocks
  cudaFuncAttributes fa;
  int dev = 0, per_sm_smem = 0, reserved = 0;
  if (cudaFuncGetAttributes(&fa, k_project_mma) != cudaSuccess || cudaGetDevice(&dev) ||
      cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) {
    cudaGetLastError();
    return 0;
  }
  const size_t per_cta = mma_smem_bytes(pr) + fa.sharedSizeBytes + (size_t)reserved;
  int per_sm = (int)((size_t)per_sm_smem / per_cta);
  per_sm = per_sm < (int)(512u / (2 * mma_tmem_cols(pr.Pp))) ? per_sm
                                                             : (int)(512u / (2 * mma_tmem_cols(pr.Pp)));
  per_sm = per_sm < 16 ? per_sm : 16;
  return per_sm * n_sm;
}

cudaError_t launch_project_mma(const Problem& pr, const Swarm& sw, const WorkTile* tiles,
                               int n_tiles, const uint16_t* posb, int grid, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  if (grid > n_tiles) grid = n_tiles;
  if (grid < 1) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3(kMmaThreads, 1, 1);
  cfg.dynamicSmemBytes = mma_smem_bytes(pr);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_project_mma, pr, sw, tiles, n_tiles, posb);
}

cudaError_t launch_merge(const Problem& pr, const Swarm& sw, int A, const EvalRes* cur2, int kp,
                         const int32_t* inv, int t, int do_update, cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)A, (unsigned)((pr.P + 7) / 8), 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_merge, pr, sw, cur2, kp, inv, t, do_update);
}

}  // namespace slm
