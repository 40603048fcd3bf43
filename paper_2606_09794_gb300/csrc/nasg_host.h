// Host-side helpers shared by the library's translation units: status
// recording, argument checks, launch geometry.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nasgabor.h"

namespace nasg {

// Records a failed CUDA call for nasg_last_cuda_error() (thread-local).
void record_cuda_error(cudaError_t e);

inline nasg_status check_launch() {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    record_cuda_error(e);
    return NASG_ERR_CUDA;
  }
  return NASG_OK;
}

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// Number of SMs of the current device (cached per device).
int sm_count();

// Device address of the library's device error word on the current device
// (resolved once per device, under a lock); nullptr if it cannot be resolved.
int* device_error_word();

// Raises `kernel`'s dynamic shared-memory limit to at least `bytes` on the current
// device. The attribute belongs to the device, so what has been set is remembered
// per (device, kernel) under a lock; later calls cost a lookup. NASG_OK or
// NASG_ERR_CUDA.
nasg_status ensure_smem_limit(const void* kernel, size_t bytes);

// Grid for a grid-stride loop over `items` with `block` threads: one item per
// thread, capped so that a 64-bit item count never overflows the grid.
inline unsigned grid_for(int64_t items, int block) {
  int64_t g = (items + block - 1) / block;
  const int64_t cap = int64_t(1) << 30;
  return static_cast<unsigned>(g < 1 ? 1 : (g > cap ? cap : g));
}

// Validates a nasg_desc; returns NASG_OK or the error.
inline nasg_status check_desc(const nasg_desc* d) {
  if (!d) return NASG_ERR_NULL;
  if (d->n < 0 || d->n_lobes < 1 || d->n_lobes > NASG_MAX_LOBES) return NASG_ERR_RANGE;
  if (d->frame_mode != NASG_FRAME_QUAT && d->frame_mode != NASG_FRAME_COS) return NASG_ERR_RANGE;
  if (d->param_dtype != NASG_DTYPE_F32 && d->param_dtype != NASG_DTYPE_BF16) return NASG_ERR_RANGE;
  if (d->norm_mode != NASG_NORM_APPROX && d->norm_mode != NASG_NORM_NONE && d->norm_mode != NASG_NORM_EXACT)
    return NASG_ERR_RANGE;
  if (d->act_mode != NASG_ACT_RAW && d->act_mode != NASG_ACT_IDENTITY) return NASG_ERR_RANGE;
  if (d->accumulate != 0 && d->accumulate != 1) return NASG_ERR_RANGE;
  if (d->lobe_family < NASG_FAMILY_NASGABOR || d->lobe_family > NASG_FAMILY_PHASE || d->reserved != 0)
    return NASG_ERR_RANGE;
  if (d->lobe_family != NASG_FAMILY_NASGABOR && d->frame_mode != NASG_FRAME_QUAT) return NASG_ERR_UNSUPPORTED;
  // element offsets are 64-bit; keep P*N*L well inside int64
  if (d->n > (int64_t(1) << 40)) return NASG_ERR_RANGE;
  return NASG_OK;
}

inline int elem_size(int32_t dtype) { return dtype == NASG_DTYPE_BF16 ? 2 : 4; }

// nasgabor_fused_fwd_bwd on the register path only (plain loads and stores, no bulk
// copies), for buffers the kernel reads and writes in page-locked host memory.
nasg_status fused_fwd_bwd_register_path(const nasg_desc* desc, const void* params, const void* c0,
                                        const float* means, const float* cam, const float* g_rgb, float* rgb,
                                        float* g_params, float* g_c0, float* g_means, cudaStream_t stream);

}  // namespace nasg
