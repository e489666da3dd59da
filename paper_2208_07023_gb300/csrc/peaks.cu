// slm_measure_peaks: the two roofs the search's kernels are held against
// that peaks measured by an HBM copy and a BF16 GEMM do not give.
//  * FP32 fused multiply-add throughput: the projection (z = X_node x_p,
//    one fmaf per feature, Sec. II-A Eq. 1) is bound by it, not by memory:
//    its rows stay in L2 across a search's iterations.
//  * L2 read bandwidth: the histogram kernels read each iteration's
//    projections, labels and multiplicities from L2, where the projection
//    just wrote them.
// Both are timed with CUDA events on the context's stream, after a warm-up
// launch, at whatever clocks the GPU runs (the caller samples them).
#include <cuda_runtime.h>

#include "slm.h"
#include "slm_internal.cuh"

namespace slm {
namespace {

constexpr int kChains = 16;   // independent FMA chains per thread
constexpr int kUnroll = 4;    // iterations per loop trip: 64 FMAs per 3 loop instructions

__global__ void __launch_bounds__(256) k_ffma_peak(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * (float)(threadIdx.x + i);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == 1234.5f) out[blockIdx.x] = s;  // keeps the chains live
}

constexpr int kL2Inflight = 4;  // 16-byte loads in flight per thread

__global__ void __launch_bounds__(256) k_l2_read(const float4* __restrict__ buf, int64_t n4,
                                                 int reps, float* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.0f;
  for (int r = 0; r < reps; ++r) {
    for (int64_t i = tid; i < n4; i += stride * kL2Inflight) {
      float4 v[kL2Inflight];
#pragma unroll
      for (int u = 0; u < kL2Inflight; ++u) {
        const int64_t j = i + u * stride;
        v[u] = j < n4 ? __ldcg(buf + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kL2Inflight; ++u) acc += v[u].x + v[u].y + v[u].z + v[u].w;
    }
  }
  if (acc == 1234.5f) out[blockIdx.x] = acc;  // keeps the loads live
}

}  // namespace
}  // namespace slm

using namespace slm;

extern "C" slm_status slm_measure_peaks(int device, void* cuda_stream, double* ffma_tflops,
                                        double* l2_read_gbs) {
  if (!ffma_tflops && !l2_read_gbs) return SLM_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
    return SLM_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int n_sm = 0;
  slm_status status = SLM_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float* out = nullptr;
  float4* buf = nullptr;
  const int64_t l2_bytes = 48ll << 20;  // fits the 129 MB L2 with room to spare
  do {
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMalloc(&out, sizeof(float) * 64 * 1024) != cudaSuccess) {
      status = SLM_ECUDA;
      break;
    }
    if (ffma_tflops) {
      // 8 blocks of 256 threads per SM: 64 warps, every FMA pipe fed
      const int blocks = 8 * n_sm, iters = 4096;
      float best_ms = 0.f;
      for (int rep = 0; rep < 4 && status == SLM_OK; ++rep) {
        cudaEventRecord(e0, st);
        k_ffma_peak<<<blocks, 256, 0, st>>>(out, iters, 0.99999994f, 1e-7f);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          status = SLM_ECUDA;
          break;
        }
        if (rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;  // rep 0 warms up
      }
      if (status != SLM_OK) break;
      const double flops = 2.0 * blocks * 256.0 * kChains * kUnroll * (double)iters;
      *ffma_tflops = flops / (best_ms * 1e-3) / 1e12;
    }
    if (l2_read_gbs) {
      if (cudaMalloc(&buf, (size_t)l2_bytes) != cudaSuccess ||
          cudaMemsetAsync(buf, 0, (size_t)l2_bytes, st) != cudaSuccess) {
        status = SLM_ECUDA;
        break;
      }
      const int64_t n4 = l2_bytes / 16;
      const int blocks = 8 * n_sm, reps = 8;
      float best_ms = 0.f;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        k_l2_read<<<blocks, 256, 0, st>>>(buf, n4, reps, out);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          status = SLM_ECUDA;
          break;
        }
        if (rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
      }
      if (status != SLM_OK) break;
      *l2_read_gbs = (double)l2_bytes * reps / (best_ms * 1e-3) / 1e9;
    }
  } while (false);
  if (cudaGetLastError() != cudaSuccess) status = SLM_ECUDA;
  if (buf) cudaFree(buf);
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaSetDevice(prev);
  return status;
}
