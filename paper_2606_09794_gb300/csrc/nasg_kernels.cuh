// NASGabor evaluation kernels (forward, backward, fused forward+backward).
//
// Mapping (warp slices): the L lobes of a primitive are taken by a slice of
// S = next_pow2(ceil(L/2)) consecutive lanes (S divides 32), lane g of the
// slice owning lobes 2g and 2g+1, evaluated together in packed FP32x2
// arithmetic (lanes past the last lobe idle). Lobe-minor storage makes the
// lobes of 32/S consecutive primitives one contiguous span of every parameter
// plane, so each plane is read (4 B bf16 / 8 B f32 per lane) and each gradient
// plane written (8 B per lane) as one contiguous warp-wide access in whole
// sectors. A thread carries two lobes' state only, which keeps registers low
// and occupancy high.
// Per-primitive sums over lobes (colour, dLoss/dd) are reduced across the slice
// with xor shuffles; the slice's first lane writes the per-primitive outputs.
// The backward recomputes every lobe quantity from the inputs; nothing is
// stored by the forward. No atomics: each output element has one writer.
#pragma once

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
  int32_t slice;        // S = next_pow2(ceil(n_lobes / 2)) lanes per primitive
  int32_t slice_log2;
  int32_t identity;
  int32_t normalised;
  int32_t accumulate;
  const float* g_rgb;
  float* rgb;
  float* g_params;
  float* g_c0;
  float* g_means;
};

template <int FRAME>
struct FrameTraits {
  static constexpr int P = (FRAME == NASG_FRAME_QUAT) ? 10 : 9;  // raw scalars per lobe
  static constexpr int B = (FRAME == NASG_FRAME_QUAT) ? 4 : 3;   // first non-frame plane
};

// Evaluates the lobes held in pv[0..P) (one lobe per component of V): adds their
// colour into rgb and, with BWD, writes the P raw-parameter gradients into gp
// and adds dLoss/dd into gd.
template <int FRAME, bool FWD, bool BWD, class V>
__device__ __forceinline__ void lobe_step(const V* pv, const V* d, const V* gc, bool identity, bool normalised,
                                          V* rgb, V* gd, V* gp) {
  constexpr int B = FrameTraits<FRAME>::B;
  Act<V> act;
  activate(pv + B, identity, act);
  V x[3], z[3];
  QuatFrame<V> qf;
  CosFrame<V> cf;
  if (FRAME == NASG_FRAME_QUAT) {
    quat_frame(pv, qf);
#pragma unroll
    for (int c = 0; c < 3; ++c) { x[c] = qf.x[c]; z[c] = qf.z[c]; }
  } else {
    cos_frame(pv, identity, cf);
#pragma unroll
    for (int c = 0; c < 3; ++c) { x[c] = cf.x[c]; z[c] = cf.z[c]; }
  }
  LobePartials<V> pd;
  const V G = lobe<BWD>(d, x, z, act.lam, act.a, act.k, normalised, &pd);
  if (FWD) {
#pragma unroll
    for (int c = 0; c < 3; ++c) rgb[c] = vfma(act.w[c], G, rgb[c]);
  }
  if (BWD) {
    const V gG = vfma(gc[0], act.w[0], vfma(gc[1], act.w[1], gc[2] * act.w[2]));
    gp[B + 0] = gG * pd.G_lam * act.s_lam;
    gp[B + 1] = gG * pd.G_a * act.s_a;
    gp[B + 2] = gG * pd.G_k * act.s_k;
#pragma unroll
    for (int c = 0; c < 3; ++c) gp[B + 3 + c] = gc[c] * G * act.s_w[c];
    const V gv = gG * pd.G_v, gu = gG * pd.G_u;
    const V gx[3] = {gv * d[0], gv * d[1], gv * d[2]};
    const V gz[3] = {gu * d[0], gu * d[1], gu * d[2]};
#pragma unroll
    for (int c = 0; c < 3; ++c) gd[c] = vfma(gu, z[c], vfma(gv, x[c], gd[c]));
    if (FRAME == NASG_FRAME_QUAT) {
      quat_frame_grad(qf, gx, gz, gp);
    } else {
      cos_frame_grad(cf, gx, gz, gp);
    }
  }
}

__device__ __forceinline__ void store1(float* p, float v, bool acc) { *p = acc ? *p + v : v; }
__device__ __forceinline__ void store2(float* p, P2 v, bool acc) {
  float2* q = reinterpret_cast<float2*>(p);
  if (acc) {
    const float2 o = *q;
    v.v.x += o.x;
    v.v.y += o.y;
  }
  *q = v.v;
}

// Raw words of one lane's work item, fetched one item ahead of the compute:
// the two lobes' P stored scalars (one 32-bit word per plane for bf16 pairs, a
// float2 for f32), the primitive's mean and upstream gradient.
template <typename T>
struct RawWord;
template <>
struct RawWord<float> {
  using type = float2;
};
template <>
struct RawWord<__nv_bfloat16> {
  using type = uint32_t;
};

template <typename T, int P>
struct RawItem {
  typename RawWord<T>::type w[P];
  float mu[3];
  float gc[3];
  int64_t i;  // primitive, -1 if none
};

template <typename T, int P, bool EVEN, bool BWD>
__device__ __forceinline__ void fetch_item(const EvalArgs& a, int64_t t, int l0, RawItem<T, P>& r) {
  const T* __restrict__ params = static_cast<const T*>(a.params);
  const int64_t total = a.n_items << a.slice_log2;
  r.i = -1;
  if (t >= total) return;
  const int64_t item = t >> a.slice_log2;
  const int64_t i = a.idx ? int64_t(__ldg(a.idx + item)) : item;
  if (i < 0 || i >= a.n) return;  // out-of-range index entries are skipped
  r.i = i;
#pragma unroll
  for (int c = 0; c < 3; ++c) r.mu[c] = __ldg(a.means + 3 * i + c);
  if (BWD) {
#pragma unroll
    for (int c = 0; c < 3; ++c) r.gc[c] = __ldg(a.g_rgb + 3 * i + c);
  }
  const int L = a.n_lobes;
  if (l0 >= L) return;
  const int64_t NL = a.n * L;
  const T* pb = params + i * L + l0;
  const bool second = l0 + 1 < L;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    if (EVEN) {
      r.w[p] = __ldg(reinterpret_cast<const typename RawWord<T>::type*>(pb + p * NL));
    } else if (sizeof(T) == 4) {
      const float lo = load1<T>(pb + p * NL);
      float2 v = make_float2(lo, second ? load1<T>(pb + p * NL + 1) : lo);
      r.w[p] = *reinterpret_cast<typename RawWord<T>::type*>(&v);
    } else {
      const uint32_t lo = *reinterpret_cast<const uint16_t*>(pb + p * NL);
      const uint32_t hi = second ? *reinterpret_cast<const uint16_t*>(pb + p * NL + 1) : lo;
      uint32_t w = lo | (hi << 16);
      r.w[p] = *reinterpret_cast<typename RawWord<T>::type*>(&w);
    }
  }
}

__device__ __forceinline__ P2 unpack(float2 w) { P2 r; r.v = w; return r; }
__device__ __forceinline__ P2 unpack(uint32_t w) { return p2(bf16_lo(w), bf16_hi(w)); }

// Each lane evaluates two lobes (2g, 2g+1) of its primitive in packed FP32x2
// arithmetic; a slice of S = next_pow2(ceil(L/2)) lanes covers the primitive.
// EVEN (L even, planes 2-element aligned): one 2-element load / store per plane.
// The grid is persistent (a few blocks per SM) and each thread fetches its next
// item's raw words before computing the current one, so that the loads of one
// item overlap the arithmetic of the previous.
template <int FRAME, typename T, int MODE, bool EVEN>
__global__ void __launch_bounds__(256, 2) eval_kernel(const EvalArgs a) {
  constexpr int P = FrameTraits<FRAME>::P;
  constexpr bool FWD = (MODE & kFwd) != 0;
  constexpr bool BWD = (MODE & kBwd) != 0;
  const int64_t n = a.n;
  const int L = a.n_lobes;
  const int64_t NL = n * L;
  const bool identity = a.identity != 0;
  const bool normalised = a.normalised != 0;
  const bool acc = a.accumulate != 0;
  const int S = a.slice;
  const int l0 = 2 * (threadIdx.x & (S - 1));
  const int64_t total = a.n_items << a.slice_log2;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  RawItem<T, P> cur, nxt;
  int64_t t0 = int64_t(blockIdx.x) * blockDim.x;
  fetch_item<T, P, EVEN, BWD>(a, t0 + threadIdx.x, l0, cur);
  // block-uniform loop: every lane of a warp reaches the shuffles below
  for (; t0 < total; t0 += stride) {
    fetch_item<T, P, EVEN, BWD>(a, t0 + stride + threadIdx.x, l0, nxt);
    const int64_t i = cur.i;
    float rgb[3] = {0.f, 0.f, 0.f};
    float gd[3] = {0.f, 0.f, 0.f};
    float d[3] = {0.f, 0.f, 1.f};
    float inv_dist = 0.f;
    if (i >= 0) {
      const float rx = cur.mu[0] - a.cam[0], ry = cur.mu[1] - a.cam[1], rz = cur.mu[2] - a.cam[2];
      inv_dist = rsqrtf(rx * rx + ry * ry + rz * rz);
      d[0] = rx * inv_dist; d[1] = ry * inv_dist; d[2] = rz * inv_dist;
      if (l0 < L) {
        const bool second = EVEN || (l0 + 1 < L);
        P2 pv[P];
#pragma unroll
        for (int p = 0; p < P; ++p) pv[p] = unpack(cur.w[p]);
        const P2 dv[3] = {p2(d[0]), p2(d[1]), p2(d[2])};
        P2 gcv[3] = {p2(0.f), p2(0.f), p2(0.f)};
        if (BWD) {
#pragma unroll
          for (int c = 0; c < 3; ++c) gcv[c] = p2(cur.gc[c]);
        }
        P2 rgbv[3] = {p2(0.f), p2(0.f), p2(0.f)};
        P2 gdv[3] = {p2(0.f), p2(0.f), p2(0.f)};
        P2 gp[P];
        lobe_step<FRAME, FWD, BWD>(pv, dv, gcv, identity, normalised, rgbv, gdv, gp);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          rgb[c] = rgbv[c].v.x + (second ? rgbv[c].v.y : 0.f);
          gd[c] = gdv[c].v.x + (second ? gdv[c].v.y : 0.f);
        }
        if (BWD) {
          float* gb = a.g_params + i * L + l0;
#pragma unroll
          for (int p = 0; p < P; ++p) {
            if (EVEN) {
              store2(gb + p * NL, gp[p], acc);
            } else {
              store1(gb + p * NL, gp[p].v.x, acc);
              if (second) store1(gb + p * NL + 1, gp[p].v.y, acc);
            }
          }
        }
      }
    }
    for (int o = S >> 1; o >= 1; o >>= 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (FWD) rgb[c] += __shfl_xor_sync(0xffffffffu, rgb[c], o);
        if (BWD) gd[c] += __shfl_xor_sync(0xffffffffu, gd[c], o);
      }
    }
    if (i >= 0 && l0 == 0) {
      if (FWD) {
        const T* __restrict__ c0 = static_cast<const T*>(a.c0);
#pragma unroll
        for (int c = 0; c < 3; ++c) a.rgb[3 * i + c] = rgb[c] + load1<T>(c0 + c * n + i);
      }
      if (BWD) {
#pragma unroll
        for (int c = 0; c < 3; ++c) store1(a.g_c0 + c * n + i, cur.gc[c], acc);
        if (a.g_means) {
          float gm[3];
          dir_grad(d, gd, inv_dist, gm);
#pragma unroll
          for (int c = 0; c < 3; ++c) store1(a.g_means + 3 * i + c, gm[c], acc);
        }
      }
    }
    cur = nxt;
  }
}

// Slice width (log2) for L lobes held two per lane: next power of two >= ceil(L/2).
inline int slice_log2(int n_lobes) {
  const int pairs = (n_lobes + 1) / 2;
  int k = 0;
  while ((1 << k) < pairs) ++k;
  return k;
}

// Persistent grid: as many blocks as fit on the device at once (occupancy
// calculator, per kernel), capped by the work.
constexpr int kEvalBlock = 256;

template <typename K>
unsigned persistent_grid(K kernel, int64_t threads, int block) {
  static int per_sm = 0;  // per kernel instantiation
  if (per_sm == 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, 0) != cudaSuccess || nb < 1) nb = 1;
    per_sm = nb;
  }
  const unsigned cap = unsigned(sm_count() * per_sm);
  const unsigned need = grid_for(threads, block);
  return need < cap ? need : cap;
}

template <int MODE, int FRAME, typename T>
nasg_status launch_frame_dtype(const EvalArgs& a, bool even, cudaStream_t s) {
  constexpr int kBlock = kEvalBlock;
  const int64_t threads = a.n_items << a.slice_log2;
  if (even) {
    auto k = eval_kernel<FRAME, T, MODE, true>;
    k<<<persistent_grid(k, threads, kBlock), kBlock, 0, s>>>(a);
  } else {
    auto k = eval_kernel<FRAME, T, MODE, false>;
    k<<<persistent_grid(k, threads, kBlock), kBlock, 0, s>>>(a);
  }
  return check_launch();
}

template <int MODE>
nasg_status launch_eval(const nasg_desc* desc, EvalArgs a, cudaStream_t s) {
  a.slice_log2 = slice_log2(desc->n_lobes);
  a.slice = 1 << a.slice_log2;
  const int es = elem_size(desc->param_dtype);
  const bool even = (desc->n_lobes % 2 == 0) && aligned(a.params, uintptr_t(2 * es)) &&
                    (a.g_params == nullptr || aligned(a.g_params, 8));
  const bool quat = desc->frame_mode == NASG_FRAME_QUAT;
  const bool bf16 = desc->param_dtype == NASG_DTYPE_BF16;
  if (quat) {
    return bf16 ? launch_frame_dtype<MODE, NASG_FRAME_QUAT, __nv_bfloat16>(a, even, s)
                : launch_frame_dtype<MODE, NASG_FRAME_QUAT, float>(a, even, s);
  }
  return bf16 ? launch_frame_dtype<MODE, NASG_FRAME_COS, __nv_bfloat16>(a, even, s)
              : launch_frame_dtype<MODE, NASG_FRAME_COS, float>(a, even, s);
}

// Each mode is instantiated in its own translation unit.
extern template nasg_status launch_eval<kFwd>(const nasg_desc*, EvalArgs, cudaStream_t);
extern template nasg_status launch_eval<kBwd>(const nasg_desc*, EvalArgs, cudaStream_t);
extern template nasg_status launch_eval<kFwdBwd>(const nasg_desc*, EvalArgs, cudaStream_t);

}  // namespace nasg
