// slm_evaluate_swarm_noalloc: swarm scoring for callers that cannot allocate
// device memory. All scratch lives in one fixed device array of this file;
// the call itself performs no cudaMalloc / cudaFree.
#include <cuda_runtime.h>
#include <limits.h>

#include <mutex>

#include "slm_internal.cuh"

namespace slm {
namespace {

// The only scratch of the no-allocation path. Every GPU that loads the library
// holds it until the process exits; every call overwrites it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SLM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};

// Device address of the scratch array on `device` (current), looked up once.
cudaError_t scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch[device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch[device]);
  return cudaSuccess;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Scratch layout of one call.
struct Layout {
  size_t xl, lab, yl, w, idx, z, zmm, pos, nodes, tiles, words, m1, m2, macc, mscale, total;
};

Layout layout(int64_t n_idx, int d, int Pp, int P, bool mse) {
  const int64_t ez = (n_idx + 3) / 4 * 4;
  const int64_t tiles = (n_idx + kTS - 1) / kTS;
  Layout l{};
  size_t o = 0;
  l.xl = o;
  o = align256(o + sizeof(float) * (size_t)n_idx * d);
  l.lab = o;
  o = align256(o + sizeof(int32_t) * (size_t)(n_idx + 16));
  l.yl = o;
  o = align256(o + sizeof(float) * (size_t)(n_idx + 16));
  l.w = o;
  o = align256(o + sizeof(uint32_t) * (size_t)(n_idx + 16));
  l.idx = o;
  o = align256(o + sizeof(int32_t) * (size_t)n_idx);
  l.z = o;
  o = align256(o + sizeof(float) * (size_t)P * (size_t)(ez > 0 ? ez : 4));
  l.zmm = o;
  o = align256(o + sizeof(int32_t) * 2 * (size_t)Pp);
  l.pos = o;
  o = align256(o + sizeof(float) * (size_t)Pp * d);
  l.nodes = o;
  o = align256(o + sizeof(NodeDesc));
  l.tiles = o;
  o = align256(o + sizeof(WorkTile) * (size_t)(tiles > 0 ? tiles : 1));
  l.words = o;  // [0] validation status, [1] kernel error word
  o = align256(o + 2 * sizeof(int32_t));
  if (mse) {  // fixed-point moments of the entries, the node's range and scales
    l.m1 = o;
    o = align256(o + sizeof(long long) * (size_t)(ez + 16));
    l.m2 = o;
    o = align256(o + sizeof(long long) * (size_t)(ez + 16));
    l.macc = o;  // weight (u64) and ordered-int range of y
    o = align256(o + 16);
    l.mscale = o;
    o = align256(o + 2 * sizeof(double));
  }
  l.total = o;
  return l;
}

// Writes the node, its tiles, the range sentinels and the status words, so
// nothing of an earlier call is read.
__global__ void k_noalloc_setup(NodeDesc* node, WorkTile* tiles, int n_tiles, int32_t n_idx,
                                int32_t* zmm, int Pp, int32_t* words) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *node = NodeDesc{0, n_idx, 0u, -1};
    words[0] = 0;
    words[1] = 0;
  }
  if (i < n_tiles) tiles[i] = WorkTile{0, i * kTS, min(kTS, n_idx - i * kTS), 0};
  if (i < Pp) {
    zmm[2 * i] = INT_MAX;
    zmm[2 * i + 1] = INT_MIN;
  }
}

__global__ void k_noalloc_iota(int32_t* idx, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) idx[i] = (int32_t)i;
}

// Makes `device` current for the call and gives the caller's current device
// back on every return path: the calling thread's device is the caller's
// state, not this library's.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = prev == device || cudaSetDevice(device) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (ok && prev >= 0) (void)cudaSetDevice(prev);
  }
};

// A pointer the kernels of `device` may read or write: device or managed
// memory visible to that device. Host memory (pageable or pinned) and other
// GPUs' memory are refused before anything is launched.
bool on_device(const void* ptr, int device) {
  if (!ptr) return true;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace
}  // namespace slm

using namespace slm;

extern "C" slm_status slm_evaluate_swarm_noalloc(int device, void* cuda_stream,
                                                 const slm_params* p, const float* X, int64_t n,
                                                 int32_t d, const int32_t* labels, const float* y,
                                                 const int32_t* sample_idx,
                                                 const uint32_t* weights, int64_t n_idx,
                                                 const float* positions, int32_t n_pos,
                                                 slm_eval* out) {
  if (!p || !X || !positions || !out || n < 1 || n > INT32_MAX || d < 1 || d > kMaxD ||
      n_pos < 1 || n_pos > kMaxParticles)
    return SLM_EINVAL;
  if (p->criterion < SLM_GINI || p->criterion > SLM_MSE || p->n_bins < 2 ||
      p->n_bins > kMaxBins || p->min_leaf < 1)
    return SLM_EINVAL;
  // the FP32 projection only: the tensor-core form needs buffers that depend
  // on the call's sizes, which this entry point does not have
  if (p->proj != SLM_PROJ_FP32 && p->proj != SLM_PROJ_BF16_TOPK) return SLM_EINVAL;
  if (p->proj == SLM_PROJ_BF16_TOPK) return SLM_EUNSUPPORTED;
  const bool mse = p->criterion == SLM_MSE;
  if (!mse && (p->n_classes < 2 || p->n_classes > kMaxClasses)) return SLM_EINVAL;
  if (!mse && (int64_t)p->n_bins * p->n_classes * 4 > kMaxHistBytesPerParticle)
    return SLM_EUNSUPPORTED;
  if (mse != (y != nullptr) || (labels != nullptr) == (y != nullptr)) return SLM_EINVAL;
  if (!sample_idx) n_idx = n;
  if (n_idx < 0 || n_idx > INT32_MAX) return SLM_EINVAL;
  if (p->criterion == SLM_GINI && n_idx >= (int64_t(1) << 22)) return SLM_EUNSUPPORTED;
  const int Pp = (n_pos + kPG - 1) / kPG * kPG;
  const Layout L = layout(n_idx, d, Pp, n_pos, mse);
  if (L.total > (size_t)SLM_NOALLOC_SCRATCH_BYTES) return SLM_EUNSUPPORTED;  // too large

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const DeviceGuard guard(device);
  if (!guard.ok) return SLM_ECUDA;
  if (!on_device(X, device) || !on_device(labels, device) || !on_device(y, device) ||
      !on_device(sample_idx, device) || !on_device(weights, device) ||
      !on_device(positions, device) || !on_device(out, device))
    return SLM_EINVAL;
  unsigned char* base = nullptr;
  if (scratch_address(device, &base) != cudaSuccess) return SLM_ECUDA;
  float* Xl = reinterpret_cast<float*>(base + L.xl);
  int32_t* lab_l = labels ? reinterpret_cast<int32_t*>(base + L.lab) : nullptr;
  float* y_l = y ? reinterpret_cast<float*>(base + L.yl) : nullptr;
  uint32_t* w_l = weights ? reinterpret_cast<uint32_t*>(base + L.w) : nullptr;
  int32_t* idx = reinterpret_cast<int32_t*>(base + L.idx);
  NodeDesc* node = reinterpret_cast<NodeDesc*>(base + L.nodes);
  WorkTile* tiles = reinterpret_cast<WorkTile*>(base + L.tiles);
  int32_t* words = reinterpret_cast<int32_t*>(base + L.words);
  const int n_tiles = (int)((n_idx + kTS - 1) / kTS);

  cudaError_t e;
  // clear what must start fresh: node, tiles, range sentinels, status words
  const int setup = n_tiles > Pp ? n_tiles : Pp;
  k_noalloc_setup<<<(setup + 255) / 256, 256, 0, st>>>(node, tiles, n_tiles, (int32_t)n_idx,
                                                       reinterpret_cast<int32_t*>(base + L.zmm),
                                                       Pp, words);
  if ((e = cudaGetLastError())) return SLM_ECUDA;
  if (!sample_idx && n_idx > 0) {
    k_noalloc_iota<<<(unsigned)((n_idx + 255) / 256), 256, 0, st>>>(idx, n_idx);
    if ((e = cudaGetLastError())) return SLM_ECUDA;
  }
  const int32_t* gidx = sample_idx ? sample_idx : idx;
  if ((e = launch_validate(labels, n, p->n_classes, sample_idx, sample_idx ? n_idx : 0, words,
                           st)))
    return SLM_ECUDA;
  int32_t bad = 0;
  if (cudaMemcpyAsync(&bad, words, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SLM_ECUDA;
  if (bad) return SLM_EINVAL;
  // rows, labels / targets and multiplicities in entry order
  if ((e = launch_gather(X, labels, y, gidx, n_idx, d, Xl, lab_l, y_l, st))) return SLM_ECUDA;
  if (weights && n_idx > 0 &&
      cudaMemcpyAsync(w_l, weights, sizeof(uint32_t) * (size_t)n_idx, cudaMemcpyDeviceToDevice,
                      st) != cudaSuccess)
    return SLM_ECUDA;
  // positions, zero-padded to whole particle groups
  float* pos = reinterpret_cast<float*>(base + L.pos);
  if (cudaMemsetAsync(pos, 0, sizeof(float) * (size_t)Pp * d, st) != cudaSuccess ||
      cudaMemcpyAsync(pos, positions, sizeof(float) * (size_t)n_pos * d, cudaMemcpyDeviceToDevice,
                      st) != cudaSuccess)
    return SLM_ECUDA;

  Problem pr{};
  pr.X = Xl;
  pr.lab = lab_l;
  pr.y = y_l;
  pr.w = w_l;
  pr.E = n_idx;
  pr.Ez = (n_idx + 3) / 4 * 4;
  pr.d = d;
  pr.crit = p->criterion;
  pr.K = mse ? 1 : p->n_classes;
  pr.B = p->n_bins;
  pr.min_leaf = p->min_leaf;
  pr.P = n_pos;
  pr.Pp = Pp;
  pr.G = Pp / kPG;
  Swarm sw{};
  sw.pos = pos;
  sw.cur = reinterpret_cast<EvalRes*>(out);
  sw.zmm = reinterpret_cast<int32_t*>(base + L.zmm);
  sw.z = reinterpret_cast<float*>(base + L.z);
  sw.err = words + 1;
  if (mse) {
    pr.m1 = reinterpret_cast<long long*>(base + L.m1);
    pr.m2 = reinterpret_cast<long long*>(base + L.m2);
    pr.mscale = reinterpret_cast<double*>(base + L.mscale);
    if (launch_mse_moments(pr, tiles, n_tiles, 1,
                           reinterpret_cast<unsigned long long*>(base + L.macc),
                           reinterpret_cast<int32_t*>(base + L.macc + 8),
                           reinterpret_cast<long long*>(base + L.m1),
                           reinterpret_cast<long long*>(base + L.m2),
                           reinterpret_cast<double*>(base + L.mscale), st) != cudaSuccess)
      return SLM_ECUDA;
  }
  if ((e = prepare_eval_kernels(pr))) return SLM_ECUDA;
  int n_sm = 1;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return SLM_ECUDA;
  if (n_tiles > 0 && (e = launch_project(pr, sw, tiles, n_tiles, 2 * n_sm, st)))
    return SLM_ECUDA;
  const int S = hist_split(pr, 1, n_idx, n_sm, hist_max_cluster(pr));
  if ((e = launch_hist_scan(pr, sw, node, 1, S, nullptr, 0, 0, st))) return SLM_ECUDA;
  int32_t err = 0;
  if (cudaMemcpyAsync(&err, words + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SLM_ECUDA;
  if (err_is_timeout(err)) return SLM_ETIMEOUT;
  return err ? SLM_ECUDA : SLM_OK;
}
