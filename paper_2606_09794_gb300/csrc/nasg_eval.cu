// C ABI entry points of the NASGabor evaluation: nasgabor_eval_fwd,
// nasgabor_eval_bwd and nasgabor_fused_fwd_bwd. Host-side validation, then one
// kernel launch (kernels in nasg_kernels.cuh; each mode is instantiated in its
// own translation unit, nasg_eval_{fwd,bwd,fused}.cu).
#include "nasg_kernels.cuh"

namespace nasg {

static void fill_common(EvalArgs& a, const nasg_desc* desc, const void* params, const float* means,
                        const float* cam) {
  a.params = params;
  a.means = means;
  a.cam[0] = cam[0];
  a.cam[1] = cam[1];
  a.cam[2] = cam[2];
  a.n = desc->n;
  a.n_lobes = desc->n_lobes;
  a.identity = desc->act_mode == NASG_ACT_IDENTITY;
  a.normalised = desc->norm_mode != NASG_NORM_NONE;
  a.exact = desc->norm_mode == NASG_NORM_EXACT;
  a.accumulate = desc->accumulate;
}

}  // namespace nasg

using namespace nasg;

extern "C" nasg_status nasgabor_eval_fwd(const nasg_desc* desc, const void* params, const void* c0,
                                         const float* means, const float* cam, const int32_t* idx,
                                         int64_t n_idx, float* rgb, void* stream) {
  nasg_status st = check_desc(desc);
  if (st != NASG_OK) return st;
  if (idx && n_idx < 0) return NASG_ERR_RANGE;
  if (desc->n == 0 || (idx && n_idx == 0)) return NASG_OK;
  if (!params || !c0 || !means || !cam || !rgb) return NASG_ERR_NULL;
  const int es = elem_size(desc->param_dtype);
  if (!aligned(params, es) || !aligned(c0, es) || !aligned(means, 4) || !aligned(rgb, 4) ||
      (idx && !aligned(idx, 4)))
    return NASG_ERR_ALIGN;
  EvalArgs a{};
  fill_common(a, desc, params, means, cam);
  a.c0 = c0;
  a.idx = idx;
  a.n_items = idx ? n_idx : desc->n;
  a.rgb = rgb;
  if (a.n_items == 0 || desc->n == 0) return NASG_OK;
  return launch_eval<kFwd>(desc, a, as_stream(stream));
}

extern "C" nasg_status nasgabor_eval_bwd(const nasg_desc* desc, const void* params, const float* means,
                                         const float* cam, const int32_t* idx, int64_t n_idx,
                                         const float* g_rgb, float* g_params, float* g_c0, float* g_means,
                                         void* stream) {
  nasg_status st = check_desc(desc);
  if (st != NASG_OK) return st;
  if (idx && n_idx < 0) return NASG_ERR_RANGE;
  if (desc->n == 0 || (idx && n_idx == 0)) return NASG_OK;
  if (!params || !means || !cam || !g_rgb || !g_params || !g_c0) return NASG_ERR_NULL;
  const int es = elem_size(desc->param_dtype);
  if (!aligned(params, es) || !aligned(means, 4) || !aligned(g_rgb, 4) || !aligned(g_params, 4) ||
      !aligned(g_c0, 4) || (g_means && !aligned(g_means, 4)) || (idx && !aligned(idx, 4)))
    return NASG_ERR_ALIGN;
  EvalArgs a{};
  fill_common(a, desc, params, means, cam);
  a.idx = idx;
  a.n_items = idx ? n_idx : desc->n;
  a.g_rgb = g_rgb;
  a.g_params = g_params;
  a.g_c0 = g_c0;
  a.g_means = g_means;
  if (a.n_items == 0 || desc->n == 0) return NASG_OK;
  return launch_eval<kBwd>(desc, a, as_stream(stream));
}

namespace nasg {
static nasg_status fused_impl(const nasg_desc* desc, const void* params, const void* c0, const float* means,
                              const float* cam, const float* g_rgb, float* rgb, float* g_params, float* g_c0,
                              float* g_means, bool no_staging, cudaStream_t stream) {
  nasg_status st = check_desc(desc);
  if (st != NASG_OK) return st;
  if (desc->n == 0) return NASG_OK;
  if (!params || !c0 || !means || !cam || !g_rgb || !rgb || !g_params || !g_c0) return NASG_ERR_NULL;
  const int es = elem_size(desc->param_dtype);
  if (!aligned(params, es) || !aligned(c0, es) || !aligned(means, 4) || !aligned(g_rgb, 4) ||
      !aligned(rgb, 4) || !aligned(g_params, 4) || !aligned(g_c0, 4) || (g_means && !aligned(g_means, 4)))
    return NASG_ERR_ALIGN;
  EvalArgs a{};
  fill_common(a, desc, params, means, cam);
  a.c0 = c0;
  a.n_items = desc->n;
  a.g_rgb = g_rgb;
  a.rgb = rgb;
  a.g_params = g_params;
  a.g_c0 = g_c0;
  a.g_means = g_means;
  a.no_staging = no_staging ? 1 : 0;
  if (desc->n == 0) return NASG_OK;
  return launch_eval<kFwdBwd>(desc, a, stream);
}

nasg_status fused_fwd_bwd_register_path(const nasg_desc* desc, const void* params, const void* c0,
                                        const float* means, const float* cam, const float* g_rgb, float* rgb,
                                        float* g_params, float* g_c0, float* g_means, cudaStream_t stream) {
  return fused_impl(desc, params, c0, means, cam, g_rgb, rgb, g_params, g_c0, g_means, true, stream);
}
}  // namespace nasg

extern "C" nasg_status nasgabor_fused_fwd_bwd(const nasg_desc* desc, const void* params, const void* c0,
                                              const float* means, const float* cam, const float* g_rgb,
                                              float* rgb, float* g_params, float* g_c0, float* g_means,
                                              void* stream) {
  return fused_impl(desc, params, c0, means, cam, g_rgb, rgb, g_params, g_c0, g_means, false, as_stream(stream));
}
