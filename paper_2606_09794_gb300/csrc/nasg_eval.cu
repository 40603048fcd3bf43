// NASGabor forward, backward and fused forward+backward kernels and their C ABI
// entry points (nasgabor_eval_fwd / nasgabor_eval_bwd / nasgabor_fused_fwd_bwd).
//
// Mapping: one thread per primitive (grid-stride), lobes walked in chunks of V
// (V = 4 when L % 4 == 0 and the planes are aligned), each plane of a chunk
// fetched with one vector load (16 B for f32, 8 B for bf16); lobe-minor
// storage makes the V lobes of one plane contiguous, so a warp reads 32
// consecutive chunks of every plane. The frame is rebuilt in registers; the
// per-primitive sums over lobes (colour, dLoss/dd) stay in registers; the
// backward recomputes every lobe quantity from the inputs (nothing is stored
// by the forward). No atomics: each output element has exactly one writer.
#include "nasg_device.cuh"
#include "nasg_host.h"

namespace nasg {

enum EvalMode { kFwd = 1, kBwd = 2, kFwdBwd = 3 };

struct EvalArgs {
  const void* params;
  const void* c0;
  const float* means;
  float cam[3];
  const int32_t* idx;
  int64_t n_items;
  int64_t n;
  int32_t n_lobes;
  int32_t identity;
  int32_t normalised;
  int32_t accumulate;
  const float* g_rgb;
  float* rgb;
  float* g_params;
  float* g_c0;
  float* g_means;
};

template <int FRAME, typename T, int V, int MODE>
__global__ void __launch_bounds__(256) eval_kernel(const EvalArgs a) {
  constexpr int P = (FRAME == NASG_FRAME_QUAT) ? 10 : 9;
  constexpr int B = (FRAME == NASG_FRAME_QUAT) ? 4 : 3;  // first non-frame plane
  constexpr bool FWD = (MODE & kFwd) != 0;
  constexpr bool BWD = (MODE & kBwd) != 0;
  const T* __restrict__ params = static_cast<const T*>(a.params);
  const T* __restrict__ c0 = static_cast<const T*>(a.c0);
  const int64_t n = a.n;
  const int L = a.n_lobes;
  const int64_t NL = n * L;
  const bool identity = a.identity != 0;
  const bool normalised = a.normalised != 0;
  const bool acc = a.accumulate != 0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < a.n_items; t += stride) {
    const int64_t i = a.idx ? int64_t(__ldg(a.idx + t)) : t;
    if (i < 0 || i >= n) continue;  // out-of-range index entries are skipped
    float d[3];
    const float inv_dist = view_dir(a.means, i, a.cam[0], a.cam[1], a.cam[2], d);
    float rgb[3] = {0.f, 0.f, 0.f};
    float gc[3] = {0.f, 0.f, 0.f};
    float gd[3] = {0.f, 0.f, 0.f};
    if (FWD) {
#pragma unroll
      for (int c = 0; c < 3; ++c) rgb[c] = load1<T>(c0 + c * n + i);
    }
    if (BWD) {
#pragma unroll
      for (int c = 0; c < 3; ++c) gc[c] = __ldg(a.g_rgb + 3 * i + c);
    }
    for (int l0 = 0; l0 < L; l0 += V) {
      const int64_t off = i * L + l0;
      float pv[P][V];
#pragma unroll
      for (int p = 0; p < P; ++p) VecLoad<T, V>::run(params + p * NL + off, pv[p]);
      float gp[P][V];
#pragma unroll
      for (int j = 0; j < V; ++j) {
        Act act;
        activate(pv[B][j], pv[B + 1][j], pv[B + 2][j], pv[B + 3][j], pv[B + 4][j], pv[B + 5][j], identity,
                 act);
        float x[3], z[3];
        QuatFrame qf;
        CosFrame cf;
        if (FRAME == NASG_FRAME_QUAT) {
          quat_frame(pv[0][j], pv[1][j], pv[2][j], pv[3][j], qf);
#pragma unroll
          for (int c = 0; c < 3; ++c) { x[c] = qf.x[c]; z[c] = qf.z[c]; }
        } else {
          cos_frame(pv[0][j], pv[1][j], pv[2][j], identity, cf);
#pragma unroll
          for (int c = 0; c < 3; ++c) { x[c] = cf.x[c]; z[c] = cf.z[c]; }
        }
        LobePartials pd;
        const float G = lobe<BWD>(d, x, z, act.lam, act.a, act.k, normalised, &pd);
        if (FWD) {
#pragma unroll
          for (int c = 0; c < 3; ++c) rgb[c] = fmaf(act.w[c], G, rgb[c]);
        }
        if (BWD) {
          const float gG = gc[0] * act.w[0] + gc[1] * act.w[1] + gc[2] * act.w[2];
          gp[B + 0][j] = gG * pd.G_lam * act.s_lam;
          gp[B + 1][j] = gG * pd.G_a * act.s_a;
          gp[B + 2][j] = gG * pd.G_k * act.s_k;
#pragma unroll
          for (int c = 0; c < 3; ++c) gp[B + 3 + c][j] = gc[c] * G * act.s_w[c];
          const float gv = gG * pd.G_v, gu = gG * pd.G_u;
          const float gx[3] = {gv * d[0], gv * d[1], gv * d[2]};
          const float gz[3] = {gu * d[0], gu * d[1], gu * d[2]};
#pragma unroll
          for (int c = 0; c < 3; ++c) gd[c] = fmaf(gu, z[c], fmaf(gv, x[c], gd[c]));
          if (FRAME == NASG_FRAME_QUAT) {
            float gq[4];
            quat_frame_grad(qf, gx, gz, gq);
#pragma unroll
            for (int c = 0; c < 4; ++c) gp[c][j] = gq[c];
          } else {
            float gcos[3];
            cos_frame_grad(cf, gx, gz, gcos);
#pragma unroll
            for (int c = 0; c < 3; ++c) gp[c][j] = gcos[c];
          }
        }
      }
      if (BWD) {
#pragma unroll
        for (int p = 0; p < P; ++p) VecStore<V>::run(a.g_params + p * NL + off, gp[p], acc);
      }
    }
    if (FWD) {
#pragma unroll
      for (int c = 0; c < 3; ++c) a.rgb[3 * i + c] = rgb[c];
    }
    if (BWD) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float* o = a.g_c0 + c * n + i;
        *o = acc ? *o + gc[c] : gc[c];
      }
      if (a.g_means) {
        float gm[3];
        dir_grad(d, gd, inv_dist, gm);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float* o = a.g_means + 3 * i + c;
          *o = acc ? *o + gm[c] : gm[c];
        }
      }
    }
  }
}

template <int MODE, int FRAME, typename T, int V>
static nasg_status launch_t(const EvalArgs& a, cudaStream_t s) {
  constexpr int kBlock = 256;
  eval_kernel<FRAME, T, V, MODE><<<grid_for(a.n_items, kBlock), kBlock, 0, s>>>(a);
  return check_launch();
}

template <int MODE>
static nasg_status launch_eval(const nasg_desc* desc, const EvalArgs& a, bool vec4, cudaStream_t s) {
  const bool quat = desc->frame_mode == NASG_FRAME_QUAT;
  const bool bf16 = desc->param_dtype == NASG_DTYPE_BF16;
#define NASG_DISPATCH_V(FR, TY)                                            \
  return vec4 ? launch_t<MODE, FR, TY, 4>(a, s) : launch_t<MODE, FR, TY, 1>(a, s)
  if (quat) {
    if (bf16) { NASG_DISPATCH_V(NASG_FRAME_QUAT, __nv_bfloat16); }
    NASG_DISPATCH_V(NASG_FRAME_QUAT, float);
  }
  if (bf16) { NASG_DISPATCH_V(NASG_FRAME_COS, __nv_bfloat16); }
  NASG_DISPATCH_V(NASG_FRAME_COS, float);
#undef NASG_DISPATCH_V
}

// Vector path: L multiple of 4, parameter planes aligned for one 4-lobe load
// (16 B f32 / 8 B bf16) and gradient planes for one 16 B store.
static bool can_vec4(const nasg_desc* desc, const void* params, const float* g_params) {
  if (desc->n_lobes % 4 != 0) return false;
  if (!aligned(params, uintptr_t(4) * elem_size(desc->param_dtype))) return false;
  if (g_params && !aligned(g_params, 16)) return false;
  return true;
}

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
  a.normalised = desc->norm_mode == NASG_NORM_APPROX;
  a.accumulate = desc->accumulate;
}

}  // namespace nasg

using namespace nasg;

extern "C" nasg_status nasgabor_eval_fwd(const nasg_desc* desc, const void* params, const void* c0,
                                         const float* means, const float* cam, const int32_t* idx,
                                         int64_t n_idx, float* rgb, void* stream) {
  nasg_status st = check_desc(desc);
  if (st != NASG_OK) return st;
  if (!params || !c0 || !means || !cam || !rgb) return NASG_ERR_NULL;
  if (idx && n_idx < 0) return NASG_ERR_RANGE;
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
  return launch_eval<kFwd>(desc, a, can_vec4(desc, params, nullptr), as_stream(stream));
}

extern "C" nasg_status nasgabor_eval_bwd(const nasg_desc* desc, const void* params, const float* means,
                                         const float* cam, const int32_t* idx, int64_t n_idx,
                                         const float* g_rgb, float* g_params, float* g_c0, float* g_means,
                                         void* stream) {
  nasg_status st = check_desc(desc);
  if (st != NASG_OK) return st;
  if (!params || !means || !cam || !g_rgb || !g_params || !g_c0) return NASG_ERR_NULL;
  if (idx && n_idx < 0) return NASG_ERR_RANGE;
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
  return launch_eval<kBwd>(desc, a, can_vec4(desc, params, g_params), as_stream(stream));
}

extern "C" nasg_status nasgabor_fused_fwd_bwd(const nasg_desc* desc, const void* params, const void* c0,
                                              const float* means, const float* cam, const float* g_rgb,
                                              float* rgb, float* g_params, float* g_c0, float* g_means,
                                              void* stream) {
  nasg_status st = check_desc(desc);
  if (st != NASG_OK) return st;
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
  if (desc->n == 0) return NASG_OK;
  return launch_eval<kFwdBwd>(desc, a, can_vec4(desc, params, g_params), as_stream(stream));
}
