// Batched persistent forward+backward over many independent scenes of uneven
// size in one launch (nasgabor_batched_prepare / _run / _autotune).
//
// A scene is one parameter set (its own N, L, camera and buffers). The prepare
// call writes a device table of the scenes and of their tile ranges into a
// caller workspace; the run call is one kernel launch (preceded, for dynamic
// scheduling, by a 4-byte counter reset), so a stream capture of it records a
// CUDA graph that can be replayed. Work items are tiles of k sub-tiles of
// I x 256/S primitives of one scene (S = lanes per primitive for that scene's L,
// I = unit_items: a thread evaluates I items of each sub-tile one after the other).
// Blocks take tiles round-robin (static) or from an atomic counter (dynamic),
// look the scene up in the shared-memory copy of the table, and evaluate the
// tile with the lobe-pair lanes of the single-scene kernels, fetching each
// lane's next sub-tile item before computing the current one. No thread waits
// on another block. A staged variant moves each sub-tile's parameter spans,
// means, upstream gradients and diffuse colours into shared memory with bulk
// copies (span plans for any N), three sub-tiles ahead (one elected producer
// thread, full/empty mbarriers, every wait bounded), for the scenes whose planes
// allow it (L >= 4), and loads the rest directly; its copy of the
// scene table sits in dynamic shared memory, sized for the batch. The autotuner times the candidate schedules on the
// caller's own prepared batch and returns the fastest.
#include <algorithm>
#include <vector>

#include "nasg_kernels.cuh"

namespace nasg {

struct SceneDev {
  EvalArgs args;       // the scene as the single-scene argument block, read in place from shared
                       // memory by the item arithmetic (no per-thread copy in registers)
  int64_t tile_begin;  // first global tile of this scene
  int64_t unit_begin;  // first global sub-tile (tile_begin x sub_tiles)
  int32_t staged;  // bit 0: parameter spans may be moved by bulk copies (even L >= 4, N L sizeof(T) % 16 == 0,
                   // 16-byte aligned planes); bit 1: the means, upstream gradients and diffuse colours
                   // too (16-byte aligned buffers, moved by span plans)
  int32_t pad;
};

constexpr int kMaxScenes = NASG_MAX_SCENES;
constexpr size_t kBatchHeader = 256;  // counter (uint32) + padding

struct BatchArgs {
  const SceneDev* table;
  uint32_t* counter;  // dynamic scheduling
  int32_t n_scenes;
  int32_t sub_tiles;  // k
  int64_t total_tiles;
  int32_t dynamic;
  int* dev_err;
};

template <typename T, int P>
__device__ __forceinline__ void fetch_scene_item(const EvalArgs& sc, int64_t prim, int l0, bool valid,
                                                 RawItem<T, P>& r) {
  r.ok = 0;
  if (!valid || prim >= sc.n) return;
  r.ok = 1;
  r.i = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) r.mu[c] = __ldg(sc.means + 3 * prim + c);
#pragma unroll
  for (int c = 0; c < 3; ++c) r.gc[c] = __ldg(sc.g_rgb + 3 * prim + c);
  const T* c0 = static_cast<const T*>(sc.c0);
#pragma unroll
  for (int c = 0; c < 3; ++c) r.c0[c] = load1<T>(c0 + c * sc.n + prim);
  const int64_t L = sc.n_lobes;
  if (l0 >= L) return;
  const int64_t NL = sc.n * L;
  const T* params = static_cast<const T*>(sc.params);
  int64_t off = prim * L + l0;
  const bool second = l0 + 1 < L;
  const bool even = (L % 2) == 0;
#pragma unroll
  for (int p = 0; p < P; ++p, off += NL) {
    if (even) {
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

// The item arithmetic of the single-scene kernels. PAIRS: every scene of the batch
// has even L, pair-aligned planes and 32-bit offsets (pair loads and stores, 32-bit
// index arithmetic); else the general form (any L, 64-bit offsets). With the default
// modes and pairs, L = 4, 8 and 16 run the arithmetic with the lobe count fixed at
// compile time (slice width and reduction bounds constants), as the single-scene
// kernel does; the scene table is ordered by lobe count, so a block's consecutive
// units (and the units all blocks work on at one time) mostly share one instance.
template <int FRAME, typename T, int FLAGS, bool PAIRS>
__device__ __forceinline__ void eval_scene_item(const EvalArgs& a, const RawItem<T, FrameTraits<FRAME>::P>& r,
                                                int64_t prim, int l0) {
  if constexpr (PAIRS && FLAGS == kFlagsDefault) {
    switch (a.n_lobes) {  // block-uniform
      case 4: eval_item<FRAME, T, uint32_t, kFwdBwd, true, FLAGS, 4>(a, r, uint32_t(prim), l0); return;
      case 8: eval_item<FRAME, T, uint32_t, kFwdBwd, true, FLAGS, 8>(a, r, uint32_t(prim), l0); return;
      case 16: eval_item<FRAME, T, uint32_t, kFwdBwd, true, FLAGS, 16>(a, r, uint32_t(prim), l0); return;
      default: break;
    }
  }
  if (PAIRS) eval_item<FRAME, T, uint32_t, kFwdBwd, true, FLAGS>(a, r, uint32_t(prim), l0);
  else eval_item<FRAME, T, int64_t, kFwdBwd, false, FLAGS>(a, r, prim, l0);
}

// Order of the scenes in the device table: by lobe-count class (4, 8, 16, others),
// then as given (the table is internal; each record holds its scene's own buffers).
inline int lobe_class(int32_t L) { return L == 4 ? 0 : (L == 8 ? 1 : (L == 16 ? 2 : 3)); }

// FLAGS: kFlagsDefault (raw activations, approximate normalisation) or
// kFlagsRuntime (modes read from the arguments).
template <int FRAME, typename T, int FLAGS, bool PAIRS>
__global__ void __launch_bounds__(256, 2) batched_kernel(const BatchArgs b) {
  constexpr int P = FrameTraits<FRAME>::P;
  __shared__ SceneDev sd[kMaxScenes];
  __shared__ int64_t next_tile;
  {
    const int words = int(b.n_scenes * sizeof(SceneDev) / sizeof(uint32_t));
    const uint32_t* src = reinterpret_cast<const uint32_t*>(b.table);
    uint32_t* dst = reinterpret_cast<uint32_t*>(sd);
    for (int j = threadIdx.x; j < words; j += blockDim.x) dst[j] = src[j];
  }
  int64_t tile = blockIdx.x;
  if (b.dynamic) {
    if (threadIdx.x == 0) next_tile = int64_t(atomicAdd(b.counter, 1u));
    __syncthreads();
    tile = next_tile;
  }
  __syncthreads();
  for (int64_t it = 1; tile < b.total_tiles; ++it) {
    // scene of this tile: last entry with tile_begin <= tile
    int lo = 0, hi = b.n_scenes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sd[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
    }
    const EvalArgs& sc = sd[lo].args;
    const int tp = 256 >> sc.slice_log2;
    const int local = threadIdx.x >> sc.slice_log2;
    const int l0 = 2 * (threadIdx.x & ((1 << sc.slice_log2) - 1));
    const int sub = b.sub_tiles * unit_items<T>();  // sub-items of tp primitives in the tile
    const int64_t base = (tile - sd[lo].tile_begin) * int64_t(tp) * sub;
    RawItem<T, P> cur, nxt;
    fetch_scene_item<T, P>(sc, base + local, l0, true, cur);
    for (int j = 0; j < sub; ++j) {
      const int64_t prim = base + int64_t(j) * tp + local;
      fetch_scene_item<T, P>(sc, prim + tp, l0, j + 1 < sub, nxt);
      eval_scene_item<FRAME, T, FLAGS, PAIRS>(sc, cur, prim, l0);
      cur = nxt;
    }
    if (b.dynamic) {
      __syncthreads();  // everyone has read next_tile of the previous claim
      if (threadIdx.x == 0) next_tile = int64_t(atomicAdd(b.counter, 1u));
      __syncthreads();
      tile = next_tile;
    } else {
      tile = blockIdx.x + it * int64_t(gridDim.x);
    }
  }
}

struct PlanDev {
  int32_t n_scenes;
  int32_t frame_mode, param_dtype, norm_mode, act_mode;
  int32_t sub_tiles;
  int64_t total_tiles;
};


// ---------------------------------------------------------------------------
// Staged variant
// ---------------------------------------------------------------------------

// Stages in flight per block.
template <typename T>
constexpr int batch_stages() { return 3; }
constexpr int kMaxBatchStages = 3;
constexpr uint32_t kUnitEnd = 0xffffffffu;

// Shared-memory metadata of one stage, written by the producer with the unit.
struct StageMeta {
  uint32_t unit;     // global sub-tile index, kUnitEnd past the last
  int32_t scene;     // scene index, -1 for an empty unit
  int32_t staged;    // bit 0: parameter spans in the stage; bit 1: means and upstream gradients too
  int32_t count;     // primitives in the unit
  int64_t p0;        // first primitive of the unit in its scene
};

// Stage layout: batch_geom<T, P>() (P parameter spans of up to I x 512 lobes, then
// the means, upstream-gradient and diffuse-colour regions of up to I x 128
// primitives): a staged sub-tile holds I x 256/S primitives x L lobes with S >= L/2
// and L >= 4 (S >= 2); the sub-tiles of scenes with fewer lobes are loaded directly.
template <typename T, int P>
__host__ __device__ inline uint32_t batch_stage_bytes() {
  return batch_geom<T, P>().stage_bytes;
}

// Producer side: record a unit in a stage and start its copies; returns whether
// copies were started (the stage then completes when their bytes have landed).
// A block's units increase, so the scene is found by advancing `sc_i` (the
// previous unit's scene); a scene's units are its sub-tiles in order, from
// tile_begin x sub_tiles, so the unit's first primitive needs no division.
template <typename T, int P>
__device__ __forceinline__ bool issue_unit(const BatchArgs& b, const SceneDev* sd, uint32_t unit, int& sc_i,
                                           StageMeta* meta, unsigned char* st, uint64_t* bar) {
  const int64_t total_units = b.total_tiles * b.sub_tiles;
  if (int64_t(unit) >= total_units) {
    meta->unit = kUnitEnd;
    meta->scene = -1;
    meta->staged = 0;
    meta->count = 0;
    meta->p0 = 0;
    mbar_arrive(bar);
    return false;
  }
  const int64_t u = int64_t(unit);
  while (sc_i + 1 < b.n_scenes && sd[sc_i + 1].unit_begin <= u) ++sc_i;
  const EvalArgs& sc = sd[sc_i].args;
  const int32_t staged = sd[sc_i].staged;
  const int64_t n = sc.n;
  const uint32_t L = uint32_t(sc.n_lobes);
  const int64_t tp = int64_t(256 >> sc.slice_log2) * unit_items<T>();
  const int64_t p0 = (u - sd[sc_i].unit_begin) * tp;
  const int64_t count = n - p0 < tp ? n - p0 : tp;
  meta->unit = unit;
  meta->scene = count > 0 ? sc_i : -1;
  meta->count = count > 0 ? int32_t(count) : 0;
  meta->p0 = p0;
  const uint32_t bytes = count > 0 ? uint32_t(count) * L * uint32_t(sizeof(T)) : 0u;
  const bool stage_p = count > 0 && (staged & 1) && (bytes % 16u) == 0u;
  const bool stage_m = stage_p && (staged & 2);
  meta->staged = (stage_p ? 1 : 0) | (stage_m ? 2 : 0);
  if (!stage_p) {
    mbar_arrive(bar);
    return false;
  }
  constexpr TileGeom g = batch_geom<T, P>();
  uint32_t total = uint32_t(P) * bytes;
  PrimPlans pp;
  if (stage_m) {
    // the plain-load parts are written first; the arrive below releases them
    pp = unit_plans<T>(uint64_t(n), uint64_t(p0), uint32_t(count));
    span_tail(st + g.off_mu, sc.means, pp.mu);
    span_tail(st + g.off_gc, sc.g_rgb, pp.mu);
    total += 2u * pp.mu.bulk;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      span_tail(st + g.off_c0 + c * g.c0_cap, sc.c0, pp.c0[c]);
      total += pp.c0[c].bulk;
    }
  }
  mbar_arrive_expect_tx(bar, total);
  // parameter plane p of the unit: plane stride N L sizeof(T) bytes, advanced by additions
  const uint64_t stride = uint64_t(n) * L * sizeof(T);
  const unsigned char* src = static_cast<const unsigned char*>(sc.params) + uint64_t(p0) * L * sizeof(T);
#pragma unroll
  for (int p = 0; p < P; ++p, src += stride) bulk_g2s(st + size_t(p) * g.plane_bytes, src, bytes, bar);
  if (stage_m) {
    if (pp.mu.bulk) {
      bulk_g2s(st + g.off_mu, reinterpret_cast<const unsigned char*>(sc.means) + pp.mu.src, pp.mu.bulk, bar);
      bulk_g2s(st + g.off_gc, reinterpret_cast<const unsigned char*>(sc.g_rgb) + pp.mu.src, pp.mu.bulk, bar);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (pp.c0[c].bulk)
        bulk_g2s(st + g.off_c0 + c * g.c0_cap, static_cast<const unsigned char*>(sc.c0) + pp.c0[c].src,
                 pp.c0[c].bulk, bar);
  }
  return true;
}

template <int FRAME, typename T, int FLAGS, bool PAIRS>
__global__ void __launch_bounds__(kStagedThreads, 2) batched_staged_kernel(const BatchArgs b) {
  constexpr int P = FrameTraits<FRAME>::P;
  constexpr int NS = batch_stages<T>();
  using W = typename RawWord<T>::type;
  __shared__ StageMeta meta[kMaxBatchStages];
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr TileGeom g = batch_geom<T, P>();
  constexpr uint32_t sbytes = g.stage_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * sbytes);
  uint64_t* empty = full + NS;
  SceneDev* sd = reinterpret_cast<SceneDev*>(empty + NS);  // the scene table (n_scenes records)
  {
    const int words = int(b.n_scenes * sizeof(SceneDev) / sizeof(uint32_t));
    const uint32_t* src = reinterpret_cast<const uint32_t*>(b.table);
    uint32_t* dst = reinterpret_cast<uint32_t*>(sd);
    for (int j = threadIdx.x; j < words; j += blockDim.x) dst[j] = src[j];
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kStagedWarps);
    }
    fence_barrier_init();
  }
  __syncthreads();
  // Producer role, rotating as in the single-scene staged kernel: the refill of
  // the stage read in iteration j is issued in iteration j + 1 by lane 0 of warp
  // j mod (warps per block). An issuing lane keeps the stages it filled that it
  // has not yet seen complete (and the parity of that phase) for the drain on
  // error, and its own scene cursor (the units it is handed increase).
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  uint32_t pending = 0, pend_par = 0;
  int issue_scene = 0;
  auto next_unit = [&](uint32_t it) -> uint32_t {
    return b.dynamic ? atomicAdd(b.counter, 1u) : uint32_t(blockIdx.x + uint64_t(it) * gridDim.x);
  };
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (issue_unit<T, P>(b, sd, next_unit(s), issue_scene, &meta[s], smem + s * sbytes, &full[s]))
        pending |= 1u << s;
  }
  bool failed = false;
  for (uint32_t it = 0;; ++it) {
    if (it >= 1 && lane == 0 && warp == (it - 1) % kStagedWarps) {
      const uint32_t pit = it - 1;
      const int ps = int(pit % NS);
      if (mbar_wait(&empty[ps], (pit / NS) & 1u, b.dev_err)) {
        fence_proxy_async();
        const uint32_t nit = pit + NS;
        if (issue_unit<T, P>(b, sd, next_unit(nit), issue_scene, &meta[ps], smem + ps * sbytes, &full[ps])) {
          pending |= 1u << ps;
          pend_par = (pend_par & ~(1u << ps)) | (((nit / NS) & 1u) << ps);
        }
      } else {
        failed = true;
      }
    }
    const int s = int(it % NS);
    const bool arrived = __all_sync(0xffffffffu, mbar_wait(&full[s], (it / NS) & 1u, b.dev_err));
    if (!arrived) {
      failed = true;
      break;  // warp-uniform; the other warps give up on their own waits
    }
    pending &= ~(1u << s);  // this stage's fill (whoever issued it) has landed
    const StageMeta m = meta[s];
    if (m.unit == kUnitEnd) break;  // block-uniform: every warp reads the same stage
    const EvalArgs& sc = sd[m.scene >= 0 ? m.scene : 0].args;
#pragma unroll
    for (int k = 0; k < unit_items<T>(); ++k) {
      RawItem<T, P> r;
      r.ok = 0;
      int64_t prim = 0;
      int l0 = 0;
      if (m.scene >= 0) {
        const int local = int(threadIdx.x) >> sc.slice_log2;
        const int loc = local + k * (256 >> sc.slice_log2);  // this item's primitive in the unit
        l0 = 2 * (int(threadIdx.x) & ((1 << sc.slice_log2) - 1));
        prim = m.p0 + loc;
        if (m.staged & 1) {
          r.ok = loc < m.count;
          if (r.ok) {
            r.i = 0;
            const unsigned char* st = smem + s * sbytes;
            if (m.staged & 2) {
              // a unit's first primitive is a multiple of 256/S >= 16: the means start
              // on a 16-byte boundary, diffuse-colour plane c at c0_head(c, N)
              const float* mu = reinterpret_cast<const float*>(st + g.off_mu);
              const float* gc = reinterpret_cast<const float*>(st + g.off_gc);
#pragma unroll
              for (int c = 0; c < 3; ++c) r.mu[c] = mu[3 * loc + c];
#pragma unroll
              for (int c = 0; c < 3; ++c) r.gc[c] = gc[3 * loc + c];
#pragma unroll
              for (int c = 0; c < 3; ++c)
                r.c0[c] = to_float(*reinterpret_cast<const T*>(st + g.off_c0 + c * g.c0_cap + c0_head<T>(c, sc.n) +
                                                               loc * sizeof(T)));
            } else {
#pragma unroll
              for (int c = 0; c < 3; ++c) r.mu[c] = __ldg(sc.means + 3 * prim + c);
#pragma unroll
              for (int c = 0; c < 3; ++c) r.gc[c] = __ldg(sc.g_rgb + 3 * prim + c);
              const T* c0 = static_cast<const T*>(sc.c0);
#pragma unroll
              for (int c = 0; c < 3; ++c) r.c0[c] = load1<T>(c0 + c * sc.n + prim);
            }
            if (l0 < sc.n_lobes) {
#pragma unroll
              for (int p = 0; p < P; ++p)
                r.w[p] = *reinterpret_cast<const W*>(st + size_t(p) * g.plane_bytes +
                                                     size_t(loc * sc.n_lobes + l0) * sizeof(T));
            }
          }
        } else {
          fetch_scene_item<T, P>(sc, prim, l0, loc < m.count, r);
        }
      }
      if (k == unit_items<T>() - 1) {
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
      }
      if (m.scene >= 0) eval_scene_item<FRAME, T, FLAGS, PAIRS>(sc, r, prim, l0);
    }
  }
  // on a failed wait, let the copies this block started finish before leaving (bounded)
  if (lane == 0 && failed) {
    for (int s = 0; s < NS; ++s)
      if (pending & (1u << s)) mbar_wait(&full[s], (pend_par >> s) & 1u, nullptr, 1u << 16);
  }
}

}  // namespace nasg

using namespace nasg;

extern "C" size_t nasgabor_batched_workspace_bytes(int32_t n_scenes) {
  if (n_scenes < 1 || n_scenes > kMaxScenes) return 0;
  return kBatchHeader + size_t(n_scenes) * sizeof(SceneDev);
}

extern "C" nasg_status nasgabor_batched_prepare(const nasg_scene* scenes, int32_t n_scenes,
                                                const nasg_batch_modes* modes, int32_t sub_tiles,
                                                void* workspace, size_t workspace_bytes, nasg_batch_plan* plan,
                                                void* stream) {
  if (!scenes || !modes || !workspace || !plan) return NASG_ERR_NULL;
  if (n_scenes < 1 || n_scenes > kMaxScenes) return NASG_ERR_RANGE;
  if (sub_tiles < 1 || sub_tiles > 64) return NASG_ERR_RANGE;
  if (workspace_bytes < nasgabor_batched_workspace_bytes(n_scenes)) return NASG_ERR_RANGE;
  if (!aligned(workspace, 16)) return NASG_ERR_ALIGN;
  if (modes->frame_mode != NASG_FRAME_QUAT && modes->frame_mode != NASG_FRAME_COS) return NASG_ERR_RANGE;
  if (modes->param_dtype != NASG_DTYPE_F32 && modes->param_dtype != NASG_DTYPE_BF16) return NASG_ERR_RANGE;
  if (modes->norm_mode != NASG_NORM_APPROX && modes->norm_mode != NASG_NORM_NONE &&
      modes->norm_mode != NASG_NORM_EXACT)
    return NASG_ERR_RANGE;
  if (modes->act_mode != NASG_ACT_RAW && modes->act_mode != NASG_ACT_IDENTITY) return NASG_ERR_RANGE;
  const int es = elem_size(modes->param_dtype);
  std::vector<SceneDev> tab(n_scenes, SceneDev{});
  std::vector<int> order(n_scenes);
  for (int j = 0; j < n_scenes; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return lobe_class(scenes[x].n_lobes) < lobe_class(scenes[y].n_lobes);
  });
  int64_t tiles = 0, prims = 0, lobes = 0;
  bool pair_path = true;
  for (int j = 0; j < n_scenes; ++j) {
    const nasg_scene& s = scenes[order[j]];
    if (s.n < 0 || s.n > (int64_t(1) << 40) || s.n_lobes < 1 || s.n_lobes > NASG_MAX_LOBES) return NASG_ERR_RANGE;
    if (s.n > 0 && (!s.params || !s.c0 || !s.means || !s.g_rgb || !s.rgb || !s.g_params || !s.g_c0))
      return NASG_ERR_NULL;
    const void* f32[] = {s.means, s.g_rgb, s.rgb, s.g_params, s.g_c0, s.g_means};
    for (const void* p : f32)
      if (p && !aligned(p, 4)) return NASG_ERR_ALIGN;
    if ((s.params && !aligned(s.params, es)) || (s.c0 && !aligned(s.c0, es))) return NASG_ERR_ALIGN;
    // pair loads need 2-element alignment when L is even
    if (s.n_lobes % 2 == 0 && s.params && !aligned(s.params, uintptr_t(2 * es))) return NASG_ERR_ALIGN;
    SceneDev& d = tab[j];
    EvalArgs& a = d.args;
    a.params = s.params;
    a.c0 = s.c0;
    a.means = s.means;
    a.cam[0] = s.cam[0];
    a.cam[1] = s.cam[1];
    a.cam[2] = s.cam[2];
    a.idx = nullptr;
    a.n_items = s.n;
    a.n = s.n;
    a.n_lobes = s.n_lobes;
    a.slice_log2 = slice_log2(s.n_lobes);
    a.slice = 1 << a.slice_log2;
    a.identity = modes->act_mode == NASG_ACT_IDENTITY;
    a.normalised = modes->norm_mode != NASG_NORM_NONE;
    a.exact = modes->norm_mode == NASG_NORM_EXACT;
    a.accumulate = 0;
    a.g_rgb = s.g_rgb;
    a.rgb = s.rgb;
    a.g_params = s.g_params;
    a.g_c0 = s.g_c0;
    a.g_means = s.g_means;
    a.dev_err = device_error_word();
    {
      const int P = nasg_param_planes(modes->frame_mode, NASG_FAMILY_NASGABOR);
      const int64_t lim = int64_t(1) << 31;
      const bool even = s.n_lobes % 2 == 0 && (!s.params || aligned(s.params, uintptr_t(2 * es))) &&
                        (!s.g_params || aligned(s.g_params, 8));
      const bool idx32 = s.n * s.n_lobes * P < lim && 3 * s.n < lim;
      pair_path = pair_path && even && idx32;
    }
    d.staged = (s.n_lobes % 2 == 0) && s.n_lobes >= 4 && s.params && aligned(s.params, 16) && (s.n * s.n_lobes * es) % 16 == 0
                   ? 1 | (aligned(s.means, 16) && aligned(s.g_rgb, 16) && aligned(s.c0, 16) ? 2 : 0)
                   : 0;
    d.tile_begin = tiles;
    d.unit_begin = tiles * sub_tiles;
    d.pad = 0;
    const int64_t tile_prims = int64_t(256 >> a.slice_log2) * unit_items_of(modes->param_dtype) * sub_tiles;
    tiles += (s.n + tile_prims - 1) / tile_prims;
    prims += s.n;
    lobes += s.n * s.n_lobes;
  }
  if (tiles >= (int64_t(1) << 32)) return NASG_ERR_RANGE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  cudaStream_t st = as_stream(stream);
  if (cudaMemsetAsync(ws, 0, kBatchHeader, st) != cudaSuccess ||
      cudaMemcpyAsync(ws + kBatchHeader, tab.data(), tab.size() * sizeof(SceneDev), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    record_cuda_error(cudaGetLastError());
    return NASG_ERR_CUDA;
  }
  plan->n_scenes = n_scenes;
  plan->frame_mode = modes->frame_mode;
  plan->param_dtype = modes->param_dtype;
  plan->norm_mode = modes->norm_mode;
  plan->act_mode = modes->act_mode;
  plan->sub_tiles = sub_tiles;
  plan->pair_path = pair_path ? 1 : 0;
  plan->reserved = 0;
  plan->total_tiles = tiles;
  plan->total_prims = prims;
  plan->total_lobes = lobes;
  plan->workspace = workspace;
  return NASG_OK;
}

namespace nasg {
// dflt: raw activations and approximate normalisation (the modes compiled in).
template <int FRAME, typename T, bool PAIRS>
static nasg_status launch_batched_k(const BatchArgs& b, int blocks_per_sm, bool staged, bool dflt, cudaStream_t s) {
  if (staged) {
    constexpr int P = FrameTraits<FRAME>::P;
    auto k = dflt ? batched_staged_kernel<FRAME, T, kFlagsDefault, PAIRS>
                  : batched_staged_kernel<FRAME, T, kFlagsRuntime, PAIRS>;
    constexpr int NS = batch_stages<T>();
    const size_t smem = size_t(NS) * batch_stage_bytes<T, P>() + 2 * NS * sizeof(uint64_t) +
                        size_t(b.n_scenes) * sizeof(SceneDev);
    if (const nasg_status e = ensure_smem_limit(reinterpret_cast<const void*>(k), smem); e != NASG_OK) return e;
    int fit = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k, kStagedThreads, smem) != cudaSuccess || fit < 1)
      fit = 1;
    const int per_sm = blocks_per_sm > 0 && blocks_per_sm < fit ? blocks_per_sm : fit;
    int64_t grid = int64_t(sm_count()) * per_sm;
    const int64_t units = b.total_tiles * b.sub_tiles;
    if (grid > units) grid = units;
    if (grid < 1) return NASG_OK;
    k<<<unsigned(grid), kStagedThreads, smem, s>>>(b);
    return check_launch();
  }
  auto k = dflt ? batched_kernel<FRAME, T, kFlagsDefault, PAIRS> : batched_kernel<FRAME, T, kFlagsRuntime, PAIRS>;
  int fit = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k, 256, 0) != cudaSuccess || fit < 1) fit = 1;
  const int per_sm = blocks_per_sm > 0 && blocks_per_sm < fit ? blocks_per_sm : fit;
  int64_t grid = int64_t(sm_count()) * per_sm;
  if (grid > b.total_tiles) grid = b.total_tiles;
  if (grid < 1) return NASG_OK;
  k<<<unsigned(grid), 256, 0, s>>>(b);
  return check_launch();
}

template <int FRAME, typename T>
static nasg_status launch_batched(const BatchArgs& b, int blocks_per_sm, bool staged, bool pairs, bool dflt,
                                  cudaStream_t s) {
  return pairs ? launch_batched_k<FRAME, T, true>(b, blocks_per_sm, staged, dflt, s)
               : launch_batched_k<FRAME, T, false>(b, blocks_per_sm, staged, dflt, s);
}
}  // namespace nasg

extern "C" nasg_status nasgabor_batched_run(const nasg_batch_plan* plan, const nasg_batch_tuning* tuning,
                                            void* stream) {
  if (!plan || !plan->workspace) return NASG_ERR_NULL;
  if (plan->n_scenes < 1 || plan->n_scenes > kMaxScenes || plan->total_tiles < 0) return NASG_ERR_RANGE;
  if (plan->total_tiles == 0) return NASG_OK;
  const int dynamic = tuning ? tuning->dynamic : 1;
  const int bps = tuning ? tuning->blocks_per_sm : 0;
  const int staged = tuning ? tuning->staged : 0;
  if (dynamic != 0 && dynamic != 1) return NASG_ERR_RANGE;
  if (staged != 0 && staged != 1) return NASG_ERR_RANGE;
  if (plan->pair_path != 0 && plan->pair_path != 1) return NASG_ERR_RANGE;
  const bool pairs = plan->pair_path != 0;
  unsigned char* ws = static_cast<unsigned char*>(plan->workspace);
  cudaStream_t st = as_stream(stream);
  BatchArgs b{};
  b.table = reinterpret_cast<const SceneDev*>(ws + kBatchHeader);
  b.counter = reinterpret_cast<uint32_t*>(ws);
  b.n_scenes = plan->n_scenes;
  b.sub_tiles = plan->sub_tiles;
  b.total_tiles = plan->total_tiles;
  b.dynamic = dynamic;
  b.dev_err = device_error_word();
  const bool dflt = plan->act_mode == NASG_ACT_RAW && plan->norm_mode == NASG_NORM_APPROX;
  if (dynamic && cudaMemsetAsync(b.counter, 0, sizeof(uint32_t), st) != cudaSuccess) return check_launch();
  const bool quat = plan->frame_mode == NASG_FRAME_QUAT;
  const bool bf16 = plan->param_dtype == NASG_DTYPE_BF16;
  if (quat) {
    return bf16 ? launch_batched<NASG_FRAME_QUAT, __nv_bfloat16>(b, bps, staged, pairs, dflt, st)
                : launch_batched<NASG_FRAME_QUAT, float>(b, bps, staged, pairs, dflt, st);
  }
  return bf16 ? launch_batched<NASG_FRAME_COS, __nv_bfloat16>(b, bps, staged, pairs, dflt, st)
              : launch_batched<NASG_FRAME_COS, float>(b, bps, staged, pairs, dflt, st);
}

extern "C" nasg_status nasgabor_batched_autotune(const nasg_scene* scenes, int32_t n_scenes,
                                                 const nasg_batch_modes* modes, void* workspace,
                                                 size_t workspace_bytes, int32_t reps, nasg_batch_plan* plan,
                                                 nasg_batch_tuning* best, float* best_ms, void* stream) {
  if (!best || !plan) return NASG_ERR_NULL;
  if (reps < 1 || reps > 1000) return NASG_ERR_RANGE;
  cudaStream_t st = as_stream(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    record_cuda_error(cudaGetLastError());
    return NASG_ERR_CUDA;
  }
  const int32_t sub_choices[] = {1, 2, 4, 8};
  const int32_t bps_choices[] = {1, 2};
  float best_t = 1e30f;
  nasg_batch_tuning best_cfg{1, 2, 1, 0};
  nasg_status status = NASG_OK;
  for (int32_t k : sub_choices) {
    nasg_batch_plan pl{};
    status = nasgabor_batched_prepare(scenes, n_scenes, modes, k, workspace, workspace_bytes, &pl, stream);
    if (status != NASG_OK) break;
    for (int32_t cfg = 0; cfg < 4 && status == NASG_OK; ++cfg) {
      const int32_t dyn = cfg & 1, staged = cfg >> 1;
      for (int32_t bps : bps_choices) {
        nasg_batch_tuning t{dyn, bps, k, staged};
        status = nasgabor_batched_run(&pl, &t, stream);  // warm-up
        if (status != NASG_OK) break;
        cudaEventRecord(e0, st);
        // every timed run is checked: a refused launch would otherwise time (almost) nothing
        // and be picked as the fastest
        for (int r = 0; r < reps && status == NASG_OK; ++r) status = nasgabor_batched_run(&pl, &t, stream);
        cudaEventRecord(e1, st);
        if (status != NASG_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          record_cuda_error(cudaGetLastError());
          status = NASG_ERR_CUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= float(reps);
        if (ms < best_t) {
          best_t = ms;
          best_cfg = t;
        }
      }
    }
    if (status != NASG_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != NASG_OK) return status;
  *best = best_cfg;
  if (best_ms) *best_ms = best_t;
  // leave the workspace prepared for the winner
  return nasgabor_batched_prepare(scenes, n_scenes, modes, best_cfg.sub_tiles, workspace, workspace_bytes, plan,
                                  stream);
}
