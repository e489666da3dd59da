// Learned swarm proposal: node statistics, a 3-layer network (bfloat16
// weights, FP32 accumulation), its loss gradient, Adam, and the seeded
// initial swarm.
//
// The network maps a node's statistics s (per-class mean offsets and feature
// variances, padded to 256 features x 20 classes + 1: 5376 inputs) to a
// direction mu (256) and 64 spread radii: h1 = relu(s W1 + b1),
// h2 = relu(h1 W2 + b2), o = h2 W3 + b3. A search seeded by it starts particle
// i at sigma (mu_hat + rho_i u_i / |u_i|) (mu_hat = mu / |mu| over the node's d
// features, rho_i = softplus(o[256 + i]), u_i uniform in [-1, 1)^d from the
// swarm stream), instead of uniformly in [-1, 1)^d (Sec. III-A's "preset
// range"). The paper has no learned proposal; this is a way to start the
// swarm near a good direction.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>

#include "device_util.cuh"
#include "philox.cuh"
#include "slm_internal.cuh"

namespace slm {
namespace {

constexpr int kD = kPropD, kK = kPropK, kIn = kPropIn, kH = kPropH, kP = kPropP, kOut = kPropOut;

// ---- node statistics ------------------------------------------------------------

__global__ void k_stats_yinit(int32_t* yr, int A) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < A) {
    yr[2 * a] = INT_MAX;
    yr[2 * a + 1] = INT_MIN;
  }
}

// Regression groups: the node's y range (ordered ints) per node.
__global__ void k_stats_yrange(Problem pr, const NodeDesc* __restrict__ nodes, int32_t* yr,
                               int splits) {
  const int a = blockIdx.x;
  const NodeDesc nd = nodes[a];
  int lo = INT_MAX, hi = INT_MIN;
  for (int64_t r = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; r < nd.seg_len;
       r += (int64_t)splits * blockDim.x) {
    const int o = f2ord(pr.y[nd.seg_start + r]);
    lo = min(lo, o);
    hi = max(hi, o);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
  }
  if ((threadIdx.x & 31) == 0 && lo != INT_MAX) {
    atomicMin(&yr[2 * a], lo);
    atomicMax(&yr[2 * a + 1], hi);
  }
}

// Group of an entry: its class, or (regression) the quarter of the node's y
// range, in float with one rounding per operation.
__device__ __forceinline__ int stat_group(const Problem& pr, int64_t e, const int32_t* yr, int a) {
  if (pr.lab) return pr.lab[e];
  const float lo = ord2f(yr[2 * a]), hi = ord2f(yr[2 * a + 1]);
  if (!(hi > lo)) return 0;
  int g = (int)floorf(__fmul_rn(4.0f, __fdiv_rn(__fsub_rn(pr.y[e], lo), __fsub_rn(hi, lo))));
  return g > 3 ? 3 : (g < 0 ? 0 : g);
}

// Grid (node, 32-feature slice, row split); warp w of a block takes rows w,
// w + 8, ... of its split. Per class: sum w (x - x0); per feature: sum w (x -
// x0), sum w (x - x0)^2, with x0 the node's first row (a shift against
// cancellation). Folded into acc[A][K + 2][d] and wk[A][K] in double.
__global__ void __launch_bounds__(256)
    k_stats_accum(Problem pr, const NodeDesc* __restrict__ nodes, const int32_t* yr, int K,
                  int splits, double* acc, double* wk) {
  __shared__ float s_acc[8][kK + 2][32];
  __shared__ float s_w[8][kK];
  const int a = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const NodeDesc nd = nodes[a];
  const int d = pr.d;
  const int j = blockIdx.y * 32 + lane;
  for (int k = 0; k < K + 2; ++k) s_acc[warp][k][lane] = 0.0f;
  if (lane < K) s_w[warp][lane] = 0.0f;
  __syncwarp();
  const float x0 = (j < d && nd.seg_len > 0) ? pr.X[(int64_t)nd.seg_start * d + j] : 0.0f;
  for (int64_t r = (int64_t)blockIdx.z * 8 + warp; r < nd.seg_len; r += (int64_t)splits * 8) {
    const int64_t e = nd.seg_start + r;
    const float w = pr.w ? (float)pr.w[e] : 1.0f;
    const int g = stat_group(pr, e, yr, a);
    if (j < d) {
      const float t = pr.X[e * d + j] - x0;
      s_acc[warp][g][lane] += w * t;
      s_acc[warp][K][lane] += w * t;
      s_acc[warp][K + 1][lane] += w * t * t;
    }
    if (lane == 0 && blockIdx.y == 0) s_w[warp][g] += w;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (K + 2) * 32; i += blockDim.x) {
    const int k = i / 32, l = i % 32, jj = blockIdx.y * 32 + l;
    if (jj >= d) continue;
    float s = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += s_acc[w][k][l];
    atomicAdd(&acc[((int64_t)a * (K + 2) + k) * d + jj], (double)s);
  }
  if (blockIdx.y == 0 && threadIdx.x < K) {
    float s = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += s_w[w][threadIdx.x];
    atomicAdd(&wk[(int64_t)a * K + threadIdx.x], (double)s);
  }
}

// stats[a][k*256 + j] = class mean offset, stats[a][20*256 + j] = variance.
__global__ void k_stats_final(int d, int K, const double* __restrict__ acc,
                              const double* __restrict__ wk, float* stats) {
  const int a = blockIdx.x;
  float* st = stats + (int64_t)a * kIn;
  const double* ac = acc + (int64_t)a * (K + 2) * d;
  double W = 0.0;
  for (int k = 0; k < K; ++k) W += wk[(int64_t)a * K + k];
  for (int i = threadIdx.x; i < kIn; i += blockDim.x) {
    const int k = i / kD, j = i % kD;
    float v = 0.0f;
    if (j < d && W > 0.0) {
      const double m = ac[(int64_t)K * d + j] / W;  // shifted mean
      if (k == kK) {
        v = (float)fmax(0.0, ac[(int64_t)(K + 1) * d + j] / W - m * m);
      } else if (k < K) {
        const double wkk = wk[(int64_t)a * K + k];
        v = wkk > 0.0 ? (float)(ac[(int64_t)k * d + j] / wkk - m) : 0.0f;
      }
    }
    st[i] = v;
  }
}

// ---- network ---------------------------------------------------------------------

__device__ __forceinline__ float ld_op(const float* p) { return *p; }
__device__ __forceinline__ float ld_op(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// C[M x N] = op(A) op(B) (+ bias, relu). op(A)(m, k) = TA ? A[k lda + m] :
// A[m lda + k]; op(B)(k, n) = TB ? B[n ldb + k] : B[k ldb + n]. 64 x 64
// tiles, 16-deep K steps through shared memory, 4 x 4 outputs per thread,
// FP32 accumulation.
template <bool TA, bool TB, typename BT, int EPI>
__global__ void __launch_bounds__(256)
    k_gemm(int M, int N, int K, const float* __restrict__ A, int lda, const BT* __restrict__ B,
           int ldb, const float* __restrict__ bias, float* __restrict__ C, int ldc) {
  __shared__ float As[16][64 + 4], Bs[16][64 + 4];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int i = threadIdx.x; i < 64 * 16; i += 256) {
      int mm, kk;
      if (TA) { mm = i % 64; kk = i / 64; } else { kk = i % 16; mm = i / 16; }
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? (TA ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k]) : 0.0f;
    }
    for (int i = threadIdx.x; i < 64 * 16; i += 256) {
      int nn, kk;
      if (TB) { kk = i % 16; nn = i / 16; } else { nn = i % 64; kk = i / 64; }
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < N && k < K)
                       ? (TB ? ld_op(B + (int64_t)n * ldb + k) : ld_op(B + (int64_t)k * ldb + n))
                       : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (EPI >= 1) v += bias[n];
      if (EPI == 2) v = fmaxf(v, 0.0f);
      C[(int64_t)m * ldc + n] = v;
    }
  }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  return s;
}

// One block (256 threads) per sample r: its loss (added into *loss, already
// divided by N) and dL/do (divided by N) in double.
__global__ void __launch_bounds__(256)
    k_mlp_loss(const float* __restrict__ O, const int32_t* __restrict__ dims,
               const float* __restrict__ targets, int N, float* dO, double* loss) {
  __shared__ double sh[8];
  const int r = blockIdx.x, j = threadIdx.x;
  const float* o = O + (int64_t)r * kOut;
  const float* a = targets + (int64_t)r * kD;
  const int d = dims[r];
  const double oj = j < d ? (double)o[j] : 0.0, aj = j < d ? (double)a[j] : 0.0;
  const double c = block_sum(oj * aj, sh);
  const double mm = block_sum(oj * oj, sh);
  const double q = mm + 1e-12, sg = c >= 0.0 ? 1.0 : -1.0;
  const double nm = sqrt(mm);
  const double mh = mm > 0.0 ? oj / nm : 0.0, uj = mh - sg * aj;
  const double delta = mm > 0.0 ? sqrt(block_sum(j < d ? uj * uj : 0.0, sh)) : 1.0;
  const double hu = block_sum(j < d ? mh * uj : 0.0, sh);
  // spread: radii i < 64 on threads 0..63
  double pin = 0.0, dld = 0.0;
  if (j < kP) {
    const double tau = (j + 0.5) / kP;
    const double x = (double)o[kD + j];
    const double rho = x > 30.0 ? x : log1p(exp(x));
    const double u = delta - rho;
    pin = u >= 0.0 ? tau * u : (tau - 1.0) * u;
    dld = (u >= 0.0 ? tau : tau - 1.0) / kP;
    const double dl_drho = (u >= 0.0 ? -tau : 1.0 - tau) / kP;
    dO[(int64_t)r * kOut + kD + j] = (float)(dl_drho / (1.0 + exp(-x)) / N);
  }
  const double spread = block_sum(pin, sh);
  const double dl_ddelta = block_sum(dld, sh);
  double g = 0.0;
  if (j < d) {
    g = -2.0 * c * aj / q + 2.0 * c * c * oj / (q * q);
    if (mm > 0.0 && delta > 0.0) g += dl_ddelta * (uj - mh * hu) / (nm * delta);
  }
  dO[(int64_t)r * kOut + j] = (float)(g / N);
  if (j == 0) atomicAdd(loss, (1.0 - c * c / q + spread / kP) / N);
}

// out[n] = sum over rows of X[rows x n_cols] column n.
__global__ void k_colsum(const float* __restrict__ X, int rows, int n_cols, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cols) return;
  float s = 0.0f;
  for (int r = 0; r < rows; ++r) s += X[(int64_t)r * n_cols + c];
  out[c] = s;
}

// dH *= (H > 0)
__global__ void k_relu_bwd(float* dH, const float* __restrict__ H, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(H[i] > 0.0f)) dH[i] = 0.0f;
}

// One Adam step (Kingma and Ba, 2015); c1 = 1 - b1^t, c2 = 1 - b2^t. wb: the
// bfloat16 copy the network computes with (null for biases).
__global__ void k_adam(float* w, float* m, float* v, const float* __restrict__ g,
                       __nv_bfloat16* wb, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  if (wb) wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* wb, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

// Glorot-uniform weights from Philox: entry i of layer L is (2u - 1) lim,
// u from counter (L, i / 4, 0, purpose 8 << 24), lane i mod 4.
__global__ void k_glorot(float* w, int64_t n, uint32_t layer, float lim, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const U4 r = philox4x32_10(layer, (uint32_t)(i >> 2), 0u, 8u << 24, (uint32_t)seed,
                             (uint32_t)(seed >> 32));
  w[i] = (2.0f * uniform24(r.v[i & 3]) - 1.0f) * lim;
}

// ---- seeded swarm ----------------------------------------------------------------

// Particle i of node uid at sigma (mu_hat + rho u / |u|), u_j = 2 U - 1 of
// the swarm stream (purpose 6, iteration 0), sigma = sqrt(d / 3) (the expected
// norm of a uniform start in [-1, 1)^d, so the start velocities keep their
// relative size; the loss is scale-invariant): one rounding per operation,
// |u| = sqrt of a sequential fused multiply-add sum of squares.
__device__ void seed_particle(uint64_t seed, uint32_t uid, int i, int d, const float* mu_hat,
                              float rho, float* pos) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  float acc = 0.0f;
  for (int q = 0; q < (d + 3) / 4; ++q) {
    const U4 r = philox4x32_10(uid, 0u, (uint32_t)i, (uint32_t)q | (6u << 24), k0, k1);
    for (int c = 0; c < 4 && 4 * q + c < d; ++c) {
      const float u = __fsub_rn(__fmul_rn(2.0f, uniform24(r.v[c])), 1.0f);
      acc = fmaf(u, u, acc);
    }
  }
  const float nrm = __fsqrt_rn(acc);
  const float sigma = __fsqrt_rn(__fdiv_rn((float)d, 3.0f));
  for (int q = 0; q < (d + 3) / 4; ++q) {
    const U4 r = philox4x32_10(uid, 0u, (uint32_t)i, (uint32_t)q | (6u << 24), k0, k1);
    for (int c = 0; c < 4 && 4 * q + c < d; ++c) {
      const int j = 4 * q + c;
      const float u = __fsub_rn(__fmul_rn(2.0f, uniform24(r.v[c])), 1.0f);
      const float qv = nrm > 0.0f ? __fdiv_rn(u, nrm) : 0.0f;
      pos[j] = __fmul_rn(sigma, __fadd_rn(mu_hat[j], __fmul_rn(rho, qv)));
    }
  }
}

__global__ void k_seed_positions(uint64_t seed, uint32_t uid, int P, int d,
                                 const float* __restrict__ mu_hat, const float* __restrict__ rho,
                                 float* pos) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) seed_particle(seed, uid, i, d, mu_hat, rho[i], pos + (int64_t)i * d);
}

// The initial swarm of each node from the network's output prop[a][OUT]:
// positions seeded around sigma mu_hat, velocities 0.1 U[-1,1) as for random
// starts, ranges / bests reset (as k_swarm_init).
__global__ void __launch_bounds__(256)
    k_swarm_seed_init(Problem pr, Swarm sw, const NodeDesc* __restrict__ nodes, SwarmCoef co,
                      const float* __restrict__ prop) {
  __shared__ float s_mu[kD];
  __shared__ float s_rho[kP];
  __shared__ double sh[8];
  const int a = blockIdx.x;
  const uint32_t uid = nodes[a].uid;
  const int d = pr.d, d4 = (d + 3) >> 2;
  const float* o = prop + (int64_t)a * kOut;
  const float oj = (int)threadIdx.x < d ? o[threadIdx.x] : 0.0f;
  const double nrm = sqrt(block_sum((double)oj * oj, sh));
  if ((int)threadIdx.x < d) s_mu[threadIdx.x] = nrm > 0.0 ? (float)(oj / nrm) : 0.0f;
  if (threadIdx.x < kP) {
    const float x = o[kD + threadIdx.x];
    s_rho[threadIdx.x] = x > 30.0f ? x : log1pf(expf(x));
  }
  __syncthreads();
  float* pos = sw.pos + (int64_t)a * pr.Pp * d;
  float* vel = sw.vel + (int64_t)a * pr.Pp * d;
  const uint32_t k0 = (uint32_t)co.seed, k1 = (uint32_t)(co.seed >> 32);
  for (int p = threadIdx.x; p < pr.Pp; p += blockDim.x) {
    if (p < pr.P) {
      seed_particle(co.seed, uid, p, d, s_mu, s_rho[p % kP], pos + (int64_t)p * d);
    } else {
      for (int j = 0; j < d; ++j) pos[(int64_t)p * d + j] = 0.0f;
    }
    int* z = sw.zmm + ((int64_t)a * pr.Pp + p) * 2;
    z[0] = INT_MAX;
    z[1] = INT_MIN;
  }
  for (int e = threadIdx.x; e < pr.Pp * d4; e += blockDim.x) {
    const int p = e / d4, q = e - p * d4;
    const U4 rv = philox4x32_10(uid, 0u, (uint32_t)p, (uint32_t)q | (kInitV << 24), k0, k1);
    for (int c = 0; c < 4; ++c) {
      const int j = 4 * q + c;
      if (j >= d) break;
      vel[(int64_t)p * d + j] =
          p < pr.P ? __fmul_rn(0.1f, __fsub_rn(__fmul_rn(2.0f, uniform24(rv.v[c])), 1.0f))
                   : 0.0f;
    }
  }
  __syncthreads();
  if (sw.posb) {
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

template <typename T>
__global__ void k_gather_rows(const T* __restrict__ src, int64_t cols, const int32_t* __restrict__ idx,
                              int b, T* dst) {
  const int r = blockIdx.y;
  const T* s = src + (int64_t)idx[r] * cols;
  T* o = dst + (int64_t)r * cols;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cols;
       c += (int64_t)gridDim.x * blockDim.x)
    o[c] = s[c];
}

__global__ void k_acc_double(double* acc, const double* __restrict__ v) { *acc += *v; }

template <bool TA, bool TB, typename BT, int EPI>
cudaError_t gemm(int M, int N, int K, const float* A, int lda, const BT* B, int ldb,
                 const float* bias, float* C, int ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
  k_gemm<TA, TB, BT, EPI><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, bias, C, ldc);
  return cudaGetLastError();
}

unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---- launchers -------------------------------------------------------------------

cudaError_t launch_node_stats(const Problem& pr, const NodeDesc* nodes, int A,
                              int64_t max_len, int K, int32_t* yr, double* acc, double* wk,
                              float* stats, int n_sm, cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  cudaError_t e;
  const int fy = (pr.d + 31) / 32;
  // row splits so that the whole batch is a few waves of CTAs
  int splits = (int)((int64_t)4 * n_sm / ((int64_t)A * fy));
  splits = splits < 1 ? 1 : splits;
  const int by_rows = (int)((max_len + 255) / 256);
  splits = splits < by_rows ? splits : (by_rows < 1 ? 1 : by_rows);
  if ((e = cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)A * (K + 2) * pr.d, st))) return e;
  if ((e = cudaMemsetAsync(wk, 0, sizeof(double) * (size_t)A * K, st))) return e;
  if (!pr.lab) {
    k_stats_yinit<<<blocks(A), 256, 0, st>>>(yr, A);
    k_stats_yrange<<<dim3((unsigned)A, (unsigned)splits), 256, 0, st>>>(pr, nodes, yr, splits);
  }
  k_stats_accum<<<dim3((unsigned)A, (unsigned)fy, (unsigned)splits), 256, 0, st>>>(
      pr, nodes, yr, K, splits, acc, wk);
  k_stats_final<<<(unsigned)A, 256, 0, st>>>(pr.d, K, acc, wk, stats);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const MlpParams& m, const float* S, int N, MlpWork w,
                               cudaStream_t st) {
  cudaError_t e;
  if ((e = gemm<false, false, __nv_bfloat16, 2>(N, kH, kIn, S, kIn, m.W1b, kH, m.b1, w.H1, kH, st)))
    return e;
  if ((e = gemm<false, false, __nv_bfloat16, 2>(N, kH, kH, w.H1, kH, m.W2b, kH, m.b2, w.H2, kH, st)))
    return e;
  return gemm<false, false, __nv_bfloat16, 1>(N, kOut, kH, w.H2, kH, m.W3b, kOut, m.b3, w.O,
                                              kOut, st);
}

cudaError_t launch_mlp_loss_grad(const MlpParams& m, const float* S, const int32_t* dims,
                                 const float* targets, int N, MlpWork w, MlpGrads g,
                                 double* loss, cudaStream_t st) {
  cudaError_t e;
  if ((e = launch_mlp_forward(m, S, N, w, st))) return e;
  if ((e = cudaMemsetAsync(loss, 0, sizeof(double), st))) return e;
  k_mlp_loss<<<(unsigned)N, 256, 0, st>>>(w.O, dims, targets, N, w.dO, loss);
  // layer 3: gW3 = H2^T dO, gb3 = colsum dO, dH2 = dO W3^T (x relu')
  if ((e = gemm<true, false, float, 0>(kH, kOut, N, w.H2, kH, w.dO, kOut, nullptr, g.W3, kOut, st)))
    return e;
  k_colsum<<<blocks(kOut), 256, 0, st>>>(w.dO, N, kOut, g.b3);
  if ((e = gemm<false, true, __nv_bfloat16, 0>(N, kH, kOut, w.dO, kOut, m.W3b, kOut, nullptr,
                                              w.dH2, kH, st)))
    return e;
  k_relu_bwd<<<blocks((int64_t)N * kH), 256, 0, st>>>(w.dH2, w.H2, (int64_t)N * kH);
  // layer 2
  if ((e = gemm<true, false, float, 0>(kH, kH, N, w.H1, kH, w.dH2, kH, nullptr, g.W2, kH, st)))
    return e;
  k_colsum<<<blocks(kH), 256, 0, st>>>(w.dH2, N, kH, g.b2);
  if ((e = gemm<false, true, __nv_bfloat16, 0>(N, kH, kH, w.dH2, kH, m.W2b, kH, nullptr, w.dH1,
                                              kH, st)))
    return e;
  k_relu_bwd<<<blocks((int64_t)N * kH), 256, 0, st>>>(w.dH1, w.H1, (int64_t)N * kH);
  // layer 1
  if ((e = gemm<true, false, float, 0>(kIn, kH, N, S, kIn, w.dH1, kH, nullptr, g.W1, kH, st)))
    return e;
  k_colsum<<<blocks(kH), 256, 0, st>>>(w.dH1, N, kH, g.b1);
  return cudaGetLastError();
}

cudaError_t launch_adam(MlpParams& m, MlpState& s, const MlpGrads& g, int t, float lr,
                        cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = (float)(1.0 - pow(0.9, t)), c2 = (float)(1.0 - pow(0.999, t));
  struct {
    float* w;
    float* m;
    float* v;
    const float* g;
    __nv_bfloat16* wb;
    int64_t n;
  } parts[6] = {{m.W1, s.mW1, s.vW1, g.W1, m.W1b, (int64_t)kIn * kH},
                {m.b1, s.mb1, s.vb1, g.b1, nullptr, kH},
                {m.W2, s.mW2, s.vW2, g.W2, m.W2b, (int64_t)kH * kH},
                {m.b2, s.mb2, s.vb2, g.b2, nullptr, kH},
                {m.W3, s.mW3, s.vW3, g.W3, m.W3b, (int64_t)kH * kOut},
                {m.b3, s.mb3, s.vb3, g.b3, nullptr, kOut}};
  for (auto& p : parts)
    k_adam<<<blocks(p.n), 256, 0, st>>>(p.w, p.m, p.v, p.g, p.wb, p.n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_mlp_sync_bf16(const MlpParams& m, cudaStream_t st) {
  k_to_bf16<<<blocks((int64_t)kIn * kH), 256, 0, st>>>(m.W1, m.W1b, (int64_t)kIn * kH);
  k_to_bf16<<<blocks((int64_t)kH * kH), 256, 0, st>>>(m.W2, m.W2b, (int64_t)kH * kH);
  k_to_bf16<<<blocks((int64_t)kH * kOut), 256, 0, st>>>(m.W3, m.W3b, (int64_t)kH * kOut);
  return cudaGetLastError();
}

cudaError_t launch_mlp_init(const MlpParams& m, uint64_t seed, cudaStream_t st) {
  cudaError_t e;
  const int64_t n1 = (int64_t)kIn * kH, n2 = (int64_t)kH * kH, n3 = (int64_t)kH * kOut;
  k_glorot<<<blocks(n1), 256, 0, st>>>(m.W1, n1, 1u, sqrtf(6.0f / (kIn + kH)), seed);
  k_glorot<<<blocks(n2), 256, 0, st>>>(m.W2, n2, 2u, sqrtf(6.0f / (kH + kH)), seed);
  k_glorot<<<blocks(n3), 256, 0, st>>>(m.W3, n3, 3u, sqrtf(6.0f / (kH + kOut)), seed);
  if ((e = cudaMemsetAsync(m.b1, 0, sizeof(float) * kH, st))) return e;
  if ((e = cudaMemsetAsync(m.b2, 0, sizeof(float) * kH, st))) return e;
  if ((e = cudaMemsetAsync(m.b3, 0, sizeof(float) * kOut, st))) return e;
  return launch_mlp_sync_bf16(m, st);
}

cudaError_t launch_gather_rows(const float* src, int64_t cols, const int32_t* idx, int b,
                               float* dst, cudaStream_t st) {
  if (b <= 0) return cudaSuccess;
  k_gather_rows<float><<<dim3(blocks(cols < 4096 ? cols : 4096), (unsigned)b), 256, 0, st>>>(
      src, cols, idx, b, dst);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const int32_t* src, int64_t cols, const int32_t* idx, int b,
                               int32_t* dst, cudaStream_t st) {
  if (b <= 0) return cudaSuccess;
  k_gather_rows<int32_t><<<dim3(blocks(cols < 4096 ? cols : 4096), (unsigned)b), 256, 0, st>>>(
      src, cols, idx, b, dst);
  return cudaGetLastError();
}

cudaError_t launch_acc_double(double* acc, const double* v, cudaStream_t st) {
  k_acc_double<<<1, 1, 0, st>>>(acc, v);
  return cudaGetLastError();
}

cudaError_t launch_seed_positions(uint64_t seed, uint32_t uid, int P, int d, const float* mu_hat,
                                  const float* rho, float* pos, cudaStream_t st) {
  if (P <= 0) return cudaSuccess;
  k_seed_positions<<<blocks(P, 64), 64, 0, st>>>(seed, uid, P, d, mu_hat, rho, pos);
  return cudaGetLastError();
}

cudaError_t launch_swarm_seed_init(const Problem& pr, const Swarm& sw, const NodeDesc* nodes,
                                   int A, SwarmCoef co, const float* prop, cudaStream_t st) {
  if (A <= 0) return cudaSuccess;
  k_swarm_seed_init<<<(unsigned)A, 256, 0, st>>>(pr, sw, nodes, co, prop);
  return cudaGetLastError();
}

}  // namespace slm
