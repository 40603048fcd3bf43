// Library-wide C ABI helpers: status strings, ABI version, CUDA error record,
// device properties cache.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "nasg_host.h"
#include "nasg_tma.cuh"

namespace nasg {

// Set by a kernel whose bounded wait gave up; see nasg_device_status().
__device__ int g_device_error = 0;

int* device_error_word() {
  static std::mutex mu;
  static int* cached[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!cached[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
    cached[dev] = static_cast<int*>(p);
  }
  return cached[dev];
}

static thread_local int32_t g_last_cuda_error = 0;

void record_cuda_error(cudaError_t e) { g_last_cuda_error = static_cast<int32_t>(e); }

nasg_status ensure_smem_limit(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> set;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return check_launch();
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = set[{dev, kernel}];
  if (bytes > have) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e != cudaSuccess) {
      record_cuda_error(e);
      return NASG_ERR_CUDA;
    }
    have = bytes;
  }
  return NASG_OK;
}

int sm_count() {
  static std::mutex mu;
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> lock(mu);
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cached[dev] = v;
  }
  return cached[dev];
}

}  // namespace nasg

extern "C" int32_t nasg_lobe_planes(int32_t frame_mode) {
  if (frame_mode == NASG_FRAME_QUAT) return 10;
  if (frame_mode == NASG_FRAME_COS) return 9;
  return -1;
}

extern "C" int32_t nasg_param_planes(int32_t frame_mode, int32_t lobe_family) {
  const int32_t frame = nasg_lobe_planes(frame_mode);
  if (frame < 0) return -1;
  switch (lobe_family) {
    case NASG_FAMILY_NASGABOR: return frame;
    case NASG_FAMILY_NASG: return frame_mode == NASG_FRAME_QUAT ? 9 : -1;
    case NASG_FAMILY_SG: return frame_mode == NASG_FRAME_QUAT ? 8 : -1;
    case NASG_FAMILY_PHASE: return frame_mode == NASG_FRAME_QUAT ? 11 : -1;
    default: return -1;
  }
}

extern "C" const char* nasg_status_string(nasg_status status) {
  switch (status) {
    case NASG_OK: return "ok";
    case NASG_ERR_NULL: return "a required pointer is NULL";
    case NASG_ERR_RANGE: return "a size, count or mode is out of range";
    case NASG_ERR_ALIGN: return "a pointer is misaligned for its element type";
    case NASG_ERR_UNSUPPORTED: return "unsupported combination of modes";
    case NASG_ERR_CUDA: return "a CUDA call or kernel launch failed";
    case NASG_ERR_DEVICE: return "a kernel reported a device-side error (bounded wait gave up)";
    case NASG_ERR_CAPACITY: return "problem larger than the fixed scratch capacity of this entry point";
    default: return "unknown status";
  }
}

extern "C" int32_t nasg_last_cuda_error(void) { return nasg::g_last_cuda_error; }

extern "C" int32_t nasg_abi_version(void) { return NASG_ABI_VERSION; }

extern "C" nasg_status nasg_device_status(void* stream) {
  int v = 0;
  cudaStream_t s = nasg::as_stream(stream);
  if (cudaMemcpyFromSymbolAsync(&v, nasg::g_device_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    nasg::record_cuda_error(cudaGetLastError());
    return NASG_ERR_CUDA;
  }
  if (v == 0) return NASG_OK;
  const int zero = 0;
  if (cudaMemcpyToSymbolAsync(nasg::g_device_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    nasg::record_cuda_error(cudaGetLastError());
    return NASG_ERR_CUDA;
  }
  return NASG_ERR_DEVICE;
}

// ---------------------------------------------------------------------------
// Diagnostic probe of the elementary functions (nasg_fastmath.cuh)
// ---------------------------------------------------------------------------
#include "nasg_fastmath.cuh"

namespace nasg {
__global__ void math_probe_kernel(int fn, const float* __restrict__ x, float* __restrict__ y,
                                  float* __restrict__ y2, int64_t n) {
  __shared__ float4 tab[kTanhEntries];
  if (fn == 3) {  // block-uniform
    fill_tanh_table(tab);
    __syncthreads();
  }
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float v = x[i];
    float a = 0.f, b = 0.f;
    if (fn == 0) {
      a = vexpm1n(v);
    } else if (fn == 1) {
      vtanh(v, a, b);
    } else if (fn == 3) {
      tanh_lookup(tab, v, a, b);
    } else {
      vsincos(v, a, b);
    }
    y[i] = a;
    if (y2) y2[i] = b;
  }
}
}  // namespace nasg

extern "C" nasg_status nasg_math_probe(int32_t fn, const float* x, float* y, float* y2, int64_t n,
                                       void* stream) {
  if (fn < 0 || fn > 3 || n < 0) return NASG_ERR_RANGE;
  if (n == 0) return NASG_OK;
  if (!x || !y || (fn > 0 && !y2)) return NASG_ERR_NULL;
  nasg::math_probe_kernel<<<nasg::grid_for(n, 256), 256, 0, nasg::as_stream(stream)>>>(fn, x, y, y2, n);
  return nasg::check_launch();
}

// ---------------------------------------------------------------------------
// Diagnostic: a bounded wait on a barrier that nothing completes
// ---------------------------------------------------------------------------
namespace nasg {
__global__ void wait_timeout_probe_kernel(int* err, uint32_t limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  // no thread arrives and no copy is issued: the phase never completes
  mbar_wait(&bar, 0, err, limit);
}
}  // namespace nasg

extern "C" nasg_status nasg_probe_wait_timeout(int32_t limit, void* stream) {
  if (limit < 1 || limit > (1 << 20)) return NASG_ERR_RANGE;
  int* err = nasg::device_error_word();
  if (!err) return NASG_ERR_CUDA;
  nasg::wait_timeout_probe_kernel<<<1, 32, 0, nasg::as_stream(stream)>>>(err, uint32_t(limit));
  return nasg::check_launch();
}

// ---------------------------------------------------------------------------
// Diagnostic: issue rate of one arithmetic pipe (microbenchmark)
// ---------------------------------------------------------------------------
namespace nasg {
constexpr int kProbeChains = 8;  // independent dependency chains per thread (latency hidden)

__global__ void __launch_bounds__(256) pipe_probe_kernel(int pipe, int64_t iters, float seed, float* out) {
  float acc[kProbeChains];
  float2 acc2[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) {
    acc[c] = seed * float(threadIdx.x + c + 1) * 1e-6f;
    acc2[c] = make_float2(acc[c], -acc[c]);
  }
  if (pipe == 0) {  // MUFU: ex2.approx, each result feeding its chain's next argument
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) acc[c] = ex2a(acc[c]) - 1.5f;
    }
  } else if (pipe == 1) {  // packed FP32x2 fused multiply-add
    const float2 m = make_float2(0.999f, 0.999f), b = make_float2(1e-3f, 1e-3f);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) acc2[c] = __ffma2_rn(acc2[c], m, b);
    }
  } else {  // scalar FP32 fused multiply-add
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) acc[c] = fmaf(acc[c], 0.999f, 1e-3f);
    }
  }
  float r = 0.f;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) r += acc[c] + acc2[c].x + acc2[c].y;
  if (r == 12345.678f) out[blockIdx.x] = r;  // keeps the chains live; never true in practice
}
}  // namespace nasg

extern "C" nasg_status nasg_pipe_probe(int32_t pipe, int64_t iters, int32_t blocks_per_sm, float* out,
                                       int64_t* ops, void* stream) {
  if (pipe < 0 || pipe > 2 || iters < 1 || iters > (int64_t(1) << 24) || blocks_per_sm < 1 || blocks_per_sm > 8)
    return NASG_ERR_RANGE;
  if (!out || !ops) return NASG_ERR_NULL;
  const int64_t blocks = int64_t(nasg::sm_count()) * blocks_per_sm;
  nasg::pipe_probe_kernel<<<unsigned(blocks), 256, 0, nasg::as_stream(stream)>>>(pipe, iters, 0.5f, out);
  // one op = one instruction's lane result: a packed FFMA2 counts as two FMAs
  *ops = blocks * 256 * iters * nasg::kProbeChains * (pipe == 1 ? 2 : 1);
  return nasg::check_launch();
}
