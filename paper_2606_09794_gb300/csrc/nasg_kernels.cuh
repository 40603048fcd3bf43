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
#include "nasg_span.h"
#include "nasg_tma.cuh"

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
  int32_t exact;        // exact normalisation (implies normalised)
  int32_t accumulate;
  int32_t no_staging;   // 1: the register path only (buffers in page-locked host memory)
  const float* g_rgb;
  float* rgb;
  float* g_params;
  float* g_c0;
  float* g_means;
  int* dev_err;         // device error word (bounded waits)
};

// Stored-lobe layout. The kernels' FRAME template parameter is a layout id,
// 4 * lobe family + frame mode, so that the NASGabor lobe keeps ids 0 (QUAT) and
// 1 (COS). Planes: the frame (4 quaternion or 3 cosine scalars), then lam, a, k,
// phi and the three weights, each where the family stores it.
static_assert(kFamNasGabor == NASG_FAMILY_NASGABOR && kFamNasg == NASG_FAMILY_NASG && kFamSg == NASG_FAMILY_SG &&
                  kFamPhase == NASG_FAMILY_PHASE,
              "family codes");
constexpr int layout_id(int frame_mode, int family) { return 4 * family + frame_mode; }

template <int FRAME>
struct FrameTraits {
  static constexpr int FAM = FRAME >> 2;
  static constexpr bool QUAT = (FRAME & 3) == NASG_FRAME_QUAT;
  using F = Family<FAM>;
  static constexpr int B = QUAT ? 4 : 3;  // first non-frame plane (lam)
  static constexpr int A = B + 1;
  static constexpr int K = B + 1 + (F::HAS_A ? 1 : 0);
  static constexpr int PH = K + (F::HAS_K ? 1 : 0);
  static constexpr int W = PH + (F::HAS_PHASE ? 1 : 0);
  static constexpr int P = W + 3;         // raw scalars per lobe
};

// A lobe evaluated at one direction: activations, frame, value and (with the
// backward) the scalar partials, kept until the upstream gradient is known.
template <int FRAME, class V>
struct LobeEval {
  Act<V> act;
  QuatFrame<V> qf;
  CosFrame<V> cf;
  V x[3], z[3];
  LobePartials<V> pd;
  V G;
};

// Evaluates the lobes held in pv[0..P) (one lobe per component of V) at d. TAB: the
// stored values are BF16 and `tab` is the block's tanh table (see tanh_lookup).
template <int FRAME, bool BWD, bool TAB = false, class V>
__device__ __forceinline__ void lobe_eval(const V* pv, const V* d, bool identity, bool normalised, bool exact,
                                          LobeEval<FRAME, V>& e, const float4* tab = nullptr) {
  using TR = FrameTraits<FRAME>;
  constexpr int B = TR::B;
  if constexpr (TR::FAM == kFamNasGabor) {
    activate<TAB>(pv + B, identity, e.act, tab);
  } else {
    activate_family<TR::FAM>(pv + B, identity, e.act);
  }
  if (TR::QUAT) {
    quat_frame(pv, e.qf);
#pragma unroll
    for (int c = 0; c < 3; ++c) { e.x[c] = e.qf.x[c]; e.z[c] = e.qf.z[c]; }
  } else {
    cos_frame(pv, identity, e.cf);
#pragma unroll
    for (int c = 0; c < 3; ++c) { e.x[c] = e.cf.x[c]; e.z[c] = e.cf.z[c]; }
  }
  // raw activations: the lam / a partials come out with respect to the stored log values
  if constexpr (TR::FAM == kFamNasGabor) {
    e.G = lobe<BWD>(d, e.x, e.z, e.act.lam, e.act.a, e.act.k, normalised, exact, !identity, &e.pd);
  } else {
    e.G = lobe_family<BWD, TR::FAM>(d, e.x, e.z, e.act.lam, e.act.a, e.act.k, e.act.phi, normalised, exact,
                                    !identity, &e.pd);
  }
}

// The backward of evaluated lobes for the upstream dLoss/dRGB gc: writes the P
// raw-parameter gradients into gp and adds dLoss/dd into gd.
template <int FRAME, class V>
__device__ __forceinline__ void lobe_grad(const LobeEval<FRAME, V>& e, const V* d, const V* gc, V* gd, V* gp) {
  using TR = FrameTraits<FRAME>;
  using F = typename TR::F;
  constexpr int B = TR::B;
  const Act<V>& act = e.act;
  const LobePartials<V>& pd = e.pd;
  const V gG = vfma(gc[0], act.w[0], vfma(gc[1], act.w[1], gc[2] * act.w[2]));
  gp[B] = gG * pd.G_lam;  // the partials are already with respect to the stored scalars
  if constexpr (F::HAS_A) gp[TR::A] = gG * pd.G_a;
  if constexpr (F::HAS_K) gp[TR::K] = gG * pd.G_k * act.s_k;
  if constexpr (F::HAS_PHASE) gp[TR::PH] = gG * pd.G_phi;
#pragma unroll
  for (int c = 0; c < 3; ++c) gp[TR::W + c] = gc[c] * e.G * act.s_w[c];
  const V gv = gG * pd.G_v, gu = gG * pd.G_u;
#pragma unroll
  for (int c = 0; c < 3; ++c) gd[c] = vfma(gu, e.z[c], vfma(gv, e.x[c], gd[c]));
  if (TR::QUAT) {
    quat_frame_grad_d(e.qf, d, gv, gu, pd.u, pd.v, gp);
  } else {
    const V gx[3] = {gv * d[0], gv * d[1], gv * d[2]};
    const V gz[3] = {gu * d[0], gu * d[1], gu * d[2]};
    cos_frame_grad(e.cf, gx, gz, gp);
  }
}

// Evaluates the lobes held in pv[0..P): adds their colour into rgb and, with
// BWD, writes the P raw-parameter gradients into gp and adds dLoss/dd into gd.
template <int FRAME, bool FWD, bool BWD, bool TAB = false, class V>
__device__ __forceinline__ void lobe_step(const V* pv, const V* d, const V* gc, bool identity, bool normalised,
                                          bool exact, V* rgb, V* gd, V* gp, const float4* tab = nullptr) {
  LobeEval<FRAME, V> e;
  lobe_eval<FRAME, BWD, TAB>(pv, d, identity, normalised, exact, e, tab);
  if (FWD) {
#pragma unroll
    for (int c = 0; c < 3; ++c) rgb[c] = vfma(e.act.w[c], e.G, rgb[c]);
  }
  if (BWD) lobe_grad<FRAME>(e, d, gc, gd, gp);
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

// The kernels that read BF16-stored NASGabor lobes take the weights' tanh from a
// shared-memory table (tanh_lookup; the bits of the evaluation but for 1 - tanh^2 of
// raw weights below 2^-13, a few ulps apart).
template <int FRAME, typename T>
constexpr bool tanh_table() { return sizeof(T) == 2 && FrameTraits<FRAME>::FAM == kFamNasGabor; }

// Raw words of one lane's work item, fetched one item ahead of the compute:
// the two lobes' P stored scalars (one 32-bit word per plane for bf16 pairs, a
// float2 for f32), the primitive's mean, upstream gradient and (first lane of
// the slice) diffuse colour.
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
  float c0[3];
  int32_t ok;   // item holds a primitive
  uint32_t i;   // primitive (IDX = uint32_t) -- see EvalItem for 64-bit
};

// Element offsets use IDX (uint32_t when P*N*L < 2^31, else uint64_t).
// `total` is the number of lane items (items << slice_log2).
template <typename T, int P, typename IDX, bool EVEN, bool FWD, bool BWD>
__device__ __forceinline__ void fetch_item(const EvalArgs& a, IDX total, IDX t, int l0, RawItem<T, P>& r,
                                           IDX& prim) {
  const T* __restrict__ params = static_cast<const T*>(a.params);
  const IDX n = IDX(a.n);
  r.ok = 0;
  if (t >= total) return;
  const IDX item = t >> a.slice_log2;
  IDX i = item;
  if (a.idx) {
    const int32_t v = __ldg(a.idx + item);
    if (v < 0) return;  // out-of-range index entries are skipped
    i = IDX(v);
  }
  if (i >= n) return;
  r.ok = 1;
  prim = i;
#pragma unroll
  for (int c = 0; c < 3; ++c) r.mu[c] = __ldg(a.means + 3 * i + c);
  if (BWD) {
#pragma unroll
    for (int c = 0; c < 3; ++c) r.gc[c] = __ldg(a.g_rgb + 3 * i + c);
  }
  if (FWD) {
    const T* __restrict__ c0 = static_cast<const T*>(a.c0);
#pragma unroll
    for (int c = 0; c < 3; ++c) r.c0[c] = load1<T>(c0 + c * n + i);
  }
  const IDX L = IDX(a.n_lobes);
  if (IDX(l0) >= L) return;
  const IDX NL = n * L;
  IDX off = i * L + IDX(l0);
  const bool second = IDX(l0) + 1 < L;
#pragma unroll
  for (int p = 0; p < P; ++p, off += NL) {
    if (EVEN) {
      r.w[p] = __ldg(reinterpret_cast<const typename RawWord<T>::type*>(params + off));
    } else if (sizeof(T) == 4) {
      const float lo = load1<T>(params + off);
      float2 v = make_float2(lo, second ? load1<T>(params + off + 1) : lo);
      r.w[p] = *reinterpret_cast<typename RawWord<T>::type*>(&v);
    } else {
      const uint32_t lo = *reinterpret_cast<const uint16_t*>(params + off);
      const uint32_t hi = second ? *reinterpret_cast<const uint16_t*>(params + off + 1) : lo;
      uint32_t w = lo | (hi << 16);
      r.w[p] = *reinterpret_cast<typename RawWord<T>::type*>(&w);
    }
  }
}

__device__ __forceinline__ P2 unpack(float2 w) { P2 r; r.v = w; return r; }
__device__ __forceinline__ P2 unpack(uint32_t w) { return p2(bf16_lo(w), bf16_hi(w)); }

// Mode flags: FLAGS < 0 reads act_mode / norm_mode / accumulate from the
// arguments at run time; FLAGS >= 0 fixes them at compile time (bit 0 identity
// activations, bit 1 unnormalised, bit 2 accumulate, bit 3 exact normalisation) so that the common mode
// (raw activations, normalised, overwrite: kFlagsDefault) carries no untaken
// predicated paths.
constexpr int kFlagsRuntime = -1;
constexpr int kFlagsDefault = 0;

template <int FLAGS>
struct Flags {
  __device__ __forceinline__ static bool identity(const EvalArgs& a) {
    return FLAGS < 0 ? a.identity != 0 : (FLAGS & 1) != 0;
  }
  __device__ __forceinline__ static bool normalised(const EvalArgs& a) {
    return FLAGS < 0 ? a.normalised != 0 : (FLAGS & 2) == 0;
  }
  __device__ __forceinline__ static bool exact(const EvalArgs& a) {
    return FLAGS < 0 ? a.exact != 0 : (FLAGS & 8) != 0;
  }
  __device__ __forceinline__ static bool accumulate(const EvalArgs& a) {
    return FLAGS < 0 ? a.accumulate != 0 : (FLAGS & 4) != 0;
  }
};

__device__ __forceinline__ float pick3(const float v[3], int c) { return c == 0 ? v[0] : (c == 1 ? v[1] : v[2]); }

// Evaluates one fetched item: the lane's two lobes, the slice reductions and the
// per-primitive outputs, whose three channels are spread over the slice's lanes.
// Lanes per primitive for L lobes held two per lane: next power of two >= ceil(L/2).
constexpr int slice_of_lobes(int L) { return L <= 2 ? 1 : 2 * slice_of_lobes((L + 1) / 2); }
constexpr int log2_of(int x) { return x <= 1 ? 0 : 1 + log2_of(x >> 1); }

// LC: the lobe count when fixed at compile time (0: read from the arguments). C0_OWN: the
// item holds only the diffuse colour of the lane's own output channel, in c0[0] (slices
// of S >= 4 lanes, where a lane writes at most channel l0/2).
template <int FRAME, typename T, typename IDX, int MODE, bool EVEN, int FLAGS, int LC = 0, bool TAB = false,
          bool C0_OWN = false>
__device__ __forceinline__ void eval_item(const EvalArgs& a, const RawItem<T, FrameTraits<FRAME>::P>& cur, IDX i,
                                          int l0, const float4* tab = nullptr) {
  constexpr int P = FrameTraits<FRAME>::P;
  constexpr bool FWD = (MODE & kFwd) != 0;
  constexpr bool BWD = (MODE & kBwd) != 0;
  const IDX n = IDX(a.n);
  const IDX L = LC ? IDX(LC) : IDX(a.n_lobes);
  // the slice width, read where it is used (a cached copy cost the batched kernels registers)
  auto S = [&]() -> int { return LC ? slice_of_lobes(LC) : a.slice; };
  const bool acc = Flags<FLAGS>::accumulate(a);
  const bool ok = cur.ok != 0;
  float rgb[3] = {0.f, 0.f, 0.f};
  float gd[3] = {0.f, 0.f, 0.f};
  float d[3] = {0.f, 0.f, 1.f};
  float inv_dist = 0.f;
  if (ok) {
    inv_dist = view_dir_rn(cur.mu, a.cam, d);
    if (IDX(l0) < L) {
      const bool second = EVEN || (IDX(l0) + 1 < L);
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
      lobe_step<FRAME, FWD, BWD, TAB>(pv, dv, gcv, Flags<FLAGS>::identity(a), Flags<FLAGS>::normalised(a),
                                      Flags<FLAGS>::exact(a), rgbv, gdv, gp, tab);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        rgb[c] = rgbv[c].v.x + (second ? rgbv[c].v.y : 0.f);
        gd[c] = gdv[c].v.x + (second ? gdv[c].v.y : 0.f);
      }
      if (BWD) {
        const IDX NL = n * L;
        IDX off = i * L + IDX(l0);
        if (acc) {
#pragma unroll
          for (int p = 0; p < P; ++p, off += NL) {
            if (EVEN) {
              store2(a.g_params + off, gp[p], true);
            } else {
              store1(a.g_params + off, gp[p].v.x, true);
              if (second) store1(a.g_params + off + 1, gp[p].v.y, true);
            }
          }
        } else {
#pragma unroll
          for (int p = 0; p < P; ++p, off += NL) {
            if (EVEN) {
              store2(a.g_params + off, gp[p], false);
            } else {
              store1(a.g_params + off, gp[p].v.x, false);
              if (second) store1(a.g_params + off + 1, gp[p].v.y, false);
            }
          }
        }
      }
    }
  }
  if (FWD && BWD && S() >= 4) {  // warp-uniform
    // Reduce-scatter over the slice: the colour and dLoss/dd partials (and the
    // partial d . dLoss/dd, linear in them) are summed so that lane c < 3 of each
    // group of four ends with channel c and lane 3 with the dot product: seven
    // shuffles in place of the twelve of an all-reduce of six values.
    const int lane = threadIdx.x & 31;
    float v[7] = {rgb[0], gd[0], rgb[1], gd[1], rgb[2], gd[2], dot3_rn(gd, d)};
    for (int o = S() >> 1; o >= 4; o >>= 1) {
#pragma unroll
      for (int k = 0; k < 7; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    const bool b1 = (lane & 2) != 0, b0 = (lane & 1) != 0;
    float k0 = b1 ? v[4] : v[0], k1 = b1 ? v[5] : v[1], k2 = b1 ? v[6] : v[2], k3 = b1 ? 0.f : v[3];
    k0 += __shfl_xor_sync(0xffffffffu, b1 ? v[0] : v[4], 2);
    k1 += __shfl_xor_sync(0xffffffffu, b1 ? v[1] : v[5], 2);
    k2 += __shfl_xor_sync(0xffffffffu, b1 ? v[2] : v[6], 2);
    k3 += __shfl_xor_sync(0xffffffffu, b1 ? v[3] : 0.f, 2);
    float e0 = b0 ? k2 : k0, e1 = b0 ? k3 : k1;
    e0 += __shfl_xor_sync(0xffffffffu, b0 ? k0 : k2, 1);
    e1 += __shfl_xor_sync(0xffffffffu, b0 ? k1 : k3, 1);
    const float dot = __shfl_sync(0xffffffffu, e0, lane | 3);
    const int c = l0 >> 1;  // this lane's channel (lane index within the slice)
    if (ok && c < 3) {
      a.rgb[3 * i + c] = e0 + (C0_OWN ? cur.c0[0] : pick3(cur.c0, c));
      store1(a.g_c0 + c * n + i, pick3(cur.gc, c), acc);
      // dLoss/dmu = (I - d d^T) dLoss/dd / |mu - cam|
      if (a.g_means) store1(a.g_means + 3 * i + c, mean_grad_rn(e1, dot, pick3(d, c), inv_dist), acc);
    }
    return;
  }
  // xor-butterfly over the slice: every lane ends with the primitive's sums
  for (int o = S() >> 1; o >= 1; o >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (FWD) rgb[c] += __shfl_xor_sync(0xffffffffu, rgb[c], o);
      if (BWD) gd[c] += __shfl_xor_sync(0xffffffffu, gd[c], o);
    }
  }
  if (ok) {
    const float dot = BWD ? dot3_rn(gd, d) : 0.f;
    for (int c = l0 >> 1; c < 3; c += S()) {
      if (FWD) a.rgb[3 * i + c] = pick3(rgb, c) + (C0_OWN ? cur.c0[0] : pick3(cur.c0, c));
      if (BWD) {
        store1(a.g_c0 + c * n + i, pick3(cur.gc, c), acc);
        // dLoss/dmu = (I - d d^T) dLoss/dd / |mu - cam|
        if (a.g_means) store1(a.g_means + 3 * i + c, mean_grad_rn(pick3(gd, c), dot, pick3(d, c), inv_dist), acc);
      }
    }
  }
}

// Each lane evaluates two lobes (2g, 2g+1) of its primitive in packed FP32x2
// arithmetic; a slice of S = next_pow2(ceil(L/2)) lanes covers the primitive.
// EVEN (L even, planes 2-element aligned): one 2-element load / store per plane.
// The grid is persistent (as many blocks as fit) and each thread fetches its
// next item's raw words before computing the current one (two buffers used in
// turn), so that the loads of one item overlap the arithmetic of the previous.
template <int FRAME, typename T, typename IDX, int MODE, bool EVEN>
__global__ void __launch_bounds__(256, 2) eval_kernel(const EvalArgs a) {
  constexpr int FLAGS = kFlagsRuntime;
  constexpr int P = FrameTraits<FRAME>::P;
  constexpr bool FWD = (MODE & kFwd) != 0;
  constexpr bool BWD = (MODE & kBwd) != 0;
  constexpr bool TAB = tanh_table<FRAME, T>();
  __shared__ float4 tab[TAB ? kTanhEntries : 1];
  if constexpr (TAB) {
    fill_tanh_table(tab);
    __syncthreads();
  }
  const int l0 = 2 * (threadIdx.x & (a.slice - 1));
  const IDX total = IDX(a.n_items) << a.slice_log2;
  const IDX stride = IDX(gridDim.x) * blockDim.x;
  RawItem<T, P> b0, b1;
  IDX i0 = 0, i1 = 0;
  IDX t0 = IDX(blockIdx.x) * blockDim.x;
  fetch_item<T, P, IDX, EVEN, FWD, BWD>(a, total, t0 + threadIdx.x, l0, b0, i0);
  // block-uniform loop: every lane of a warp reaches the shuffles
  while (t0 < total) {
    fetch_item<T, P, IDX, EVEN, FWD, BWD>(a, total, t0 + stride + threadIdx.x, l0, b1, i1);
    eval_item<FRAME, T, IDX, MODE, EVEN, FLAGS, 0, TAB>(a, b0, i0, l0, tab);
    t0 += stride;
    if (t0 >= total) break;
    fetch_item<T, P, IDX, EVEN, FWD, BWD>(a, total, t0 + stride + threadIdx.x, l0, b0, i0);
    eval_item<FRAME, T, IDX, MODE, EVEN, FLAGS, 0, TAB>(a, b1, i1, l0, tab);
    t0 += stride;
  }
}

// ---------------------------------------------------------------------------
// TMA-staged variant: tiles of TP = THREADS/S consecutive primitives. For a tile,
// every parameter plane is one contiguous span of TP*L elements, and the means,
// upstream gradients and diffuse colours are contiguous too, so one elected
// thread moves a whole tile into shared memory with bulk asynchronous copies
// (cp.async.bulk) completing on the stage's "full" mbarrier. kStages tiles are
// in flight per block; each warp reads its lanes' words from the stage and
// arrives on the stage's "empty" mbarrier; one iteration later the elected
// thread waits for that stage to be empty and refills it with the tile kStages
// ahead. No block-wide barrier is taken inside the loop, and every wait is
// bounded. Requirements (checked on the host): no index list, L even,
// N L sizeof(T) a multiple of 16 bytes, 16-byte aligned buffers, 32-bit
// offsets. Any N otherwise: the spans of the means, upstream gradients and
// diffuse colours are moved by span plans (rounded to 16-byte boundaries, the
// last bytes of a buffer by plain loads).
// ---------------------------------------------------------------------------
constexpr int kStages = 3;
// Threads (and warps) of a block of the staged kernels; the launches use exactly this.
// A compile-time warp count keeps the producer's turn (iteration mod warps) cheap:
// the same modulo by blockDim.x / 32 at run time cost 3.5 % of the fused pass.
// The forward alone (fewer registers) runs 384 threads, 24 warps per SM at two
// blocks: 3 % faster than 256 for the FP32 forward with one item per thread, while
// the passes with a backward need the registers of 256-thread blocks (at 384 they
// spill).
// A tile of THREADS/S primitives is a multiple of 8 for S <= THREADS/8.
constexpr uint32_t kStagedThreads = 256;
constexpr uint32_t kStagedWarps = kStagedThreads / 32;
// (A forward that takes several items per thread and stage runs 256-thread blocks, whose
// stages of two items fit two blocks per SM.)
template <int MODE, int KI = 1>
constexpr uint32_t staged_threads() { return MODE == kFwd && KI == 1 ? 384u : kStagedThreads; }
// The full and empty barriers of the stages, rounded to 16 bytes.
constexpr uint32_t barrier_bytes(int stages) { return (2u * uint32_t(stages) * 8u + 15u) & ~15u; }
constexpr uint32_t kBarrierBytes = barrier_bytes(kStages);

// Moves the plain-load part of a span plan (the last bytes of a buffer).
__device__ __forceinline__ void span_tail(unsigned char* dst, const void* base, const SpanPlan& s) {
  if (s.tail == 0) return;
  const uint16_t* src = reinterpret_cast<const uint16_t*>(static_cast<const unsigned char*>(base) + s.src + s.bulk);
  uint16_t* d = reinterpret_cast<uint16_t*>(dst + s.bulk);
  for (uint32_t j = 0; j < s.tail / 2u; ++j) d[j] = src[j];
}

// One tile's copies, issued by one elected thread (the plans of tile_span): the
// plain-load tails first (released by the arrive), then the announcement of the
// tile's bulk bytes, then the bulk copies. (Issuing them from the 32 lanes of a
// warp side by side measured slower: the whole warp then waits on the stage.)
template <typename T, int P, bool FWD, bool BWD, bool ANYN>
__device__ __forceinline__ void issue_tile(const EvalArgs& a, const TileGeom& g, uint32_t L, uint32_t tile,
                                           unsigned char* st, uint64_t* bar) {
  const uint32_t n = uint32_t(a.n);
  const uint32_t p0 = tile * g.tp;
  const uint32_t bp = tile_span<T, P, ANYN>(g, n, L, tile, 0).bulk;  // every parameter plane's span
  const SpanPlan pm = tile_span<T, P, ANYN>(g, n, L, tile, P);
  SpanPlan pc[3];
  uint32_t total = P * bp + (BWD ? 2u : 1u) * pm.bulk;
  if (ANYN) {
    span_tail(st + g.off_mu, a.means, pm);
    if (BWD) span_tail(st + g.off_gc, a.g_rgb, pm);
  }
  if (FWD) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pc[c] = tile_span<T, P, ANYN>(g, n, L, tile, P + 2 + c);
      if (ANYN) span_tail(st + g.off_c0 + c * g.c0_cap, a.c0, pc[c]);
      total += pc[c].bulk;
    }
  }
  mbar_arrive_expect_tx(bar, total);
  const T* params = static_cast<const T*>(a.params);
  const uint32_t NL = n * L;
#pragma unroll
  for (int p = 0; p < P; ++p) bulk_g2s(st + p * g.plane_bytes, params + p * NL + p0 * L, bp, bar);
  if (pm.bulk) {
    bulk_g2s(st + g.off_mu, reinterpret_cast<const unsigned char*>(a.means) + pm.src, pm.bulk, bar);
    if (BWD) bulk_g2s(st + g.off_gc, reinterpret_cast<const unsigned char*>(a.g_rgb) + pm.src, pm.bulk, bar);
  }
  if (FWD) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (pc[c].bulk)
        bulk_g2s(st + g.off_c0 + c * g.c0_cap, static_cast<const unsigned char*>(a.c0) + pc[c].src, pc[c].bulk, bar);
  }
}

// KI: items per thread and stage (a tile of KI x THREADS/S primitives; a thread evaluates
// its KI items of a stage one after the other, which spreads the per-stage work -- the
// waits, the producer's turn, the tile arithmetic -- over KI items).
template <int FRAME, typename T, int MODE, int FLAGS, bool ANYN, int LC, int KI = 1, int NS = kStages>
__global__ void __launch_bounds__(staged_threads<MODE, KI>(), 2) eval_tma_kernel(const EvalArgs a) {
  constexpr int P = FrameTraits<FRAME>::P;
  constexpr bool FWD = (MODE & kFwd) != 0;
  constexpr bool BWD = (MODE & kBwd) != 0;
  constexpr uint32_t NT = staged_threads<MODE, KI>();
  constexpr uint32_t NW = NT / 32;
  // several items per thread at L >= 8 (S >= 4): each lane reads only its own channel's c0
  constexpr bool C0_OWN = KI > 1 && LC >= 8;
  using W = typename RawWord<T>::type;
  extern __shared__ __align__(128) unsigned char smem[];
  const int slog = LC ? log2_of(slice_of_lobes(LC)) : a.slice_log2;
  const uint32_t L = LC ? uint32_t(LC) : uint32_t(a.n_lobes);
  const TileGeom g = tile_geom<T, P, ANYN>(slog, int(L), NT * KI);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * g.stage_bytes);  // tile landed
  uint64_t* empty = full + NS;                                             // tile read by all warps
  constexpr bool TAB = tanh_table<FRAME, T>();
  // after the barriers, on a 16-byte boundary (the stages are 128-byte multiples)
  float4* tab = reinterpret_cast<float4*>(smem + NS * g.stage_bytes + barrier_bytes(NS));
  if constexpr (TAB) fill_tanh_table(tab);
  const uint32_t n = uint32_t(a.n);
  const uint32_t n_tiles = (n + g.tp - 1) / g.tp;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NW);
    }
    fence_barrier_init();
  }
  __syncthreads();
  // Producer role: the refill of the stage read in iteration j is issued, in
  // iteration j + 1, by lane 0 of warp j mod (warps per block), so the copy work
  // rotates over the warps (and the SM's sub-partitions) instead of loading one
  // warp. Each issuing lane remembers the stages it filled that it has not yet
  // seen complete (and the parity of that phase), to let them land on an error.
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  uint32_t pending = 0, pend_par = 0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const uint32_t tile = blockIdx.x + s * gridDim.x;
      if (tile < n_tiles) {
        issue_tile<T, P, FWD, BWD, ANYN>(a, g, L, tile, smem + s * g.stage_bytes, &full[s]);
        pending |= 1u << s;
      }
    }
  }
  const uint32_t local = threadIdx.x >> slog;
  const int l0 = 2 * (threadIdx.x & ((1 << slog) - 1));
  for (uint32_t it = 0;; ++it) {
    const uint32_t tile = blockIdx.x + it * gridDim.x;
    if (tile >= n_tiles) break;  // block-uniform
    // producer: refill the stage read in the previous iteration (one iteration
    // of slack, so the wait for its last reader is normally already over)
    if (it >= 1 && lane == 0 && warp == (it - 1) % NW) {
      const uint32_t pit = it - 1;
      const uint32_t nit = pit + NS;
      const uint32_t next = blockIdx.x + nit * gridDim.x;
      const int ps = pit % NS;
      if (next < n_tiles && mbar_wait(&empty[ps], (pit / NS) & 1u, a.dev_err)) {
        fence_proxy_async();
        issue_tile<T, P, FWD, BWD, ANYN>(a, g, L, next, smem + ps * g.stage_bytes, &full[ps]);
        pending |= 1u << ps;
        pend_par = (pend_par & ~(1u << ps)) | (((nit / NS) & 1u) << ps);
      }
    }
    const int s = it % NS;
    const unsigned char* st = smem + s * g.stage_bytes;
    const bool arrived = __all_sync(0xffffffffu, mbar_wait(&full[s], (it / NS) & 1u, a.dev_err));
    if (!arrived) {  // warp-uniform; the other warps give up on their own waits
      // let the copies this lane started land before the block leaves (bounded)
      if (lane == 0) {
        for (int q = 0; q < NS; ++q)
          if (pending & (1u << q)) mbar_wait(&full[q], (pend_par >> q) & 1u, nullptr, 1u << 16);
      }
      return;
    }
    pending &= ~(1u << s);  // this stage's fill (whoever issued it) has landed
    const uint32_t p0 = tile * g.tp;
    const uint32_t count = min(g.tp, n - p0);
#pragma unroll
    for (int k = 0; k < KI; ++k) {
      const uint32_t loc = local + uint32_t(k) * (NT >> slog);  // this item's primitive in the tile
      RawItem<T, P> r;
      r.ok = loc < count;
      const uint32_t i = p0 + loc;
      if (r.ok) {
        const float* mu = reinterpret_cast<const float*>(st + g.off_mu);
#pragma unroll
        for (int c = 0; c < 3; ++c) r.mu[c] = mu[3 * loc + c];
        if (BWD) {
          const float* gc = reinterpret_cast<const float*>(st + g.off_gc);
#pragma unroll
          for (int c = 0; c < 3; ++c) r.gc[c] = gc[3 * loc + c];
        }
        if (FWD) {
          // plain shared-memory reads (load1 uses the global read-only path)
          if constexpr (C0_OWN) {
            const uint32_t c = min(uint32_t(l0) >> 1, 2u);  // the lane's output channel
            r.c0[0] = to_float(*reinterpret_cast<const T*>(st + g.off_c0 + c * g.c0_cap + c0_head<T, ANYN>(c, n) +
                                                           loc * sizeof(T)));
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c)
              r.c0[c] = to_float(*reinterpret_cast<const T*>(st + g.off_c0 + c * g.c0_cap + c0_head<T, ANYN>(c, n) +
                                                             loc * sizeof(T)));
          }
        }
        if (uint32_t(l0) < L) {
#pragma unroll
          for (int p = 0; p < P; ++p)
            r.w[p] = *reinterpret_cast<const W*>(st + p * g.plane_bytes + (loc * L + l0) * sizeof(T));
        }
      }
      if (k == KI - 1) {
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
      }
      eval_item<FRAME, T, uint32_t, MODE, true, FLAGS, LC, TAB, C0_OWN>(a, r, i, l0, tab);
    }
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

template <int MODE, int FRAME, typename T, typename IDX>
nasg_status launch_idx(const EvalArgs& a, bool even, cudaStream_t s) {
  constexpr int kBlock = kEvalBlock;
  const int64_t threads = a.n_items << a.slice_log2;
  if (even) {
    auto k = eval_kernel<FRAME, T, IDX, MODE, true>;
    k<<<persistent_grid(k, threads, kBlock), kBlock, 0, s>>>(a);
  } else {
    auto k = eval_kernel<FRAME, T, IDX, MODE, false>;
    k<<<persistent_grid(k, threads, kBlock), kBlock, 0, s>>>(a);
  }
  return check_launch();
}

// The TMA-staged kernel applies (see its requirements above).
template <int MODE, int FRAME, typename T>
bool tma_eligible(const EvalArgs& a, bool even) {
  if (!even || a.idx != nullptr || a.n_items != a.n || a.no_staging) return false;
  if (uint32_t(a.slice) > staged_threads<MODE>() / 8) return false;  // tiles of a multiple of 8 primitives
  if (a.n * a.n_lobes * int64_t(sizeof(T)) % 16 != 0) return false;  // parameter planes on 16-byte boundaries
  if (a.n * a.n_lobes * FrameTraits<FRAME>::P >= (int64_t(1) << 31)) return false;
  const void* ptrs[] = {a.params, a.means, a.c0, a.g_rgb};
  for (const void* p : ptrs)
    if (p && !aligned(p, 16)) return false;
  return true;
}

template <int MODE, int FRAME, typename T, int FLAGS, bool ANYN, int LC, int KI = 1, int NS = kStages>
nasg_status launch_tma_geom(const EvalArgs& a, cudaStream_t s) {
  constexpr int P = FrameTraits<FRAME>::P;
  constexpr uint32_t NT = staged_threads<MODE, KI>();
  const TileGeom g = tile_geom<T, P, ANYN>(a.slice_log2, a.n_lobes, NT * KI);
  const size_t smem = size_t(NS) * g.stage_bytes + barrier_bytes(NS) + (tanh_table<FRAME, T>() ? kTanhBytes : 0u);
  auto k = eval_tma_kernel<FRAME, T, MODE, FLAGS, ANYN, LC, KI, NS>;
  if (const nasg_status e = ensure_smem_limit(reinterpret_cast<const void*>(k), smem); e != NASG_OK) return e;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const uint32_t n_tiles = uint32_t((a.n + g.tp - 1) / g.tp);
  const uint32_t cap = uint32_t(sm_count() * per_sm);
  k<<<n_tiles < cap ? n_tiles : cap, NT, smem, s>>>(a);
  return check_launch();
}

// N % 8 == 0: packed stages and exact spans; any other N: span plans. With the
// default modes, L = 4, 8 and 16 run instances with the lobe count (and so the
// slice width and the stage geometry) fixed at compile time (BF16 parameters,
// and the FP32 forward).
template <int MODE, int FRAME, typename T, int FLAGS, int LC>
nasg_status launch_tma_lc(const EvalArgs& a, cudaStream_t s) {
  // BF16 forward+backward: several items per thread and stage in two stages (L = 8, 16:
  // three items, tiles of 1536 lobes; L = 4: two items, tiles of 1024 lobes), which with
  // the tanh table still fit two blocks per SM; the FP32 forward alone: two items per
  // thread in two stages of 256-thread blocks (at 384 threads they would not fit two blocks)
  constexpr bool many = sizeof(T) == 2 && MODE == kFwdBwd;
  constexpr bool ffwd = sizeof(T) == 4 && MODE == kFwd;
  constexpr int KI = many ? (LC >= 8 ? 3 : 2) : (ffwd ? 2 : 1);
  constexpr int NS = (many || ffwd) ? 2 : kStages;
  return a.n % 8 == 0 ? launch_tma_geom<MODE, FRAME, T, FLAGS, false, LC, KI, NS>(a, s)
                      : launch_tma_geom<MODE, FRAME, T, FLAGS, true, LC, KI, NS>(a, s);
}

template <int MODE, int FRAME, typename T, int FLAGS>
nasg_status launch_tma(const EvalArgs& a, cudaStream_t s) {
  // (FP32 parameters with a backward: the fixed-L instances measured slower, so not used)
  if constexpr (FLAGS == kFlagsDefault && (sizeof(T) == 2 || MODE == kFwd)) {
    if (a.n_lobes == 8) return launch_tma_lc<MODE, FRAME, T, FLAGS, 8>(a, s);
    if (a.n_lobes == 4) return launch_tma_lc<MODE, FRAME, T, FLAGS, 4>(a, s);
    if (a.n_lobes == 16) return launch_tma_lc<MODE, FRAME, T, FLAGS, 16>(a, s);
  }
  return a.n % 8 == 0 ? launch_tma_geom<MODE, FRAME, T, FLAGS, false, 0>(a, s)
                      : launch_tma_geom<MODE, FRAME, T, FLAGS, true, 0>(a, s);
}

template <int MODE, int FRAME, typename T>
nasg_status launch_frame_dtype(const EvalArgs& a, bool even, cudaStream_t s) {
  if (tma_eligible<MODE, FRAME, T>(a, even)) {
    const bool dflt = a.identity == 0 && a.normalised != 0 && a.exact == 0 && a.accumulate == 0;
    return dflt ? launch_tma<MODE, FRAME, T, kFlagsDefault>(a, s) : launch_tma<MODE, FRAME, T, kFlagsRuntime>(a, s);
  }
  // 32-bit element offsets when every offset the kernel forms (P*N*L elements,
  // 3*N, and the thread index including one stride of prefetch) stays below 2^31.
  const int64_t NL = a.n * a.n_lobes;
  const int64_t threads = a.n_items << a.slice_log2;
  const int64_t lim = int64_t(1) << 31;
  const bool idx32 = NL * FrameTraits<FRAME>::P < lim && 3 * a.n < lim && 2 * threads + (int64_t(1) << 24) < lim;
  return idx32 ? launch_idx<MODE, FRAME, T, uint32_t>(a, even, s) : launch_idx<MODE, FRAME, T, uint64_t>(a, even, s);
}

// Lobe families other than NASGabor (QUAT frames): the staged kernel with
// run-time mode flags where it applies, else the register path with 64-bit
// offsets. Instantiated per family in nasg_family_{nasg,sg,phase}.cu.
template <int MODE, int FAM>
nasg_status launch_family(const EvalArgs& a, bool even, bool bf16, cudaStream_t s) {
  constexpr int LAYOUT = layout_id(NASG_FRAME_QUAT, FAM);
  if (bf16) {
    if (tma_eligible<MODE, LAYOUT, __nv_bfloat16>(a, even)) return launch_tma<MODE, LAYOUT, __nv_bfloat16, kFlagsRuntime>(a, s);
    return launch_idx<MODE, LAYOUT, __nv_bfloat16, uint64_t>(a, even, s);
  }
  if (tma_eligible<MODE, LAYOUT, float>(a, even)) return launch_tma<MODE, LAYOUT, float, kFlagsRuntime>(a, s);
  return launch_idx<MODE, LAYOUT, float, uint64_t>(a, even, s);
}

#define NASG_FAMILY_EXTERN(FAM)                                                                     \
  extern template nasg_status launch_family<kFwd, FAM>(const EvalArgs&, bool, bool, cudaStream_t);   \
  extern template nasg_status launch_family<kBwd, FAM>(const EvalArgs&, bool, bool, cudaStream_t);   \
  extern template nasg_status launch_family<kFwdBwd, FAM>(const EvalArgs&, bool, bool, cudaStream_t);
NASG_FAMILY_EXTERN(kFamNasg)
NASG_FAMILY_EXTERN(kFamSg)
NASG_FAMILY_EXTERN(kFamPhase)
#undef NASG_FAMILY_EXTERN

template <int MODE>
nasg_status launch_eval(const nasg_desc* desc, EvalArgs a, cudaStream_t s) {
  a.dev_err = device_error_word();
  a.slice_log2 = slice_log2(desc->n_lobes);
  a.slice = 1 << a.slice_log2;
  const int es = elem_size(desc->param_dtype);
  const bool even = (desc->n_lobes % 2 == 0) && aligned(a.params, uintptr_t(2 * es)) &&
                    (a.g_params == nullptr || aligned(a.g_params, 8));
  const bool quat = desc->frame_mode == NASG_FRAME_QUAT;
  const bool bf16 = desc->param_dtype == NASG_DTYPE_BF16;
  switch (desc->lobe_family) {
    case NASG_FAMILY_NASG: return launch_family<MODE, kFamNasg>(a, even, bf16, s);
    case NASG_FAMILY_SG: return launch_family<MODE, kFamSg>(a, even, bf16, s);
    case NASG_FAMILY_PHASE: return launch_family<MODE, kFamPhase>(a, even, bf16, s);
    default: break;
  }
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
