// Batched persistent forward+backward over many independent scenes of uneven
// size in one launch (nasgabor_batched_prepare / _run / _autotune).
//
// A scene is one parameter set (its own N, L, camera and buffers). The prepare
// call writes a device table of the scenes and of their tile ranges into a
// caller workspace; the run call is one kernel launch (preceded, for dynamic
// scheduling, by a 4-byte counter reset), so a stream capture of it records a
// CUDA graph that can be replayed. Work items are tiles of k sub-tiles of
// 256/S primitives of one scene (S = lanes per primitive for that scene's L).
// Blocks take tiles round-robin (static) or from an atomic counter (dynamic),
// look the scene up in the shared-memory copy of the table, and evaluate the
// tile with the lobe-pair lanes of the single-scene kernels, fetching each
// lane's next sub-tile item before computing the current one. No thread waits
// on another block. A staged variant moves each sub-tile's parameter spans,
// means and upstream gradients into shared memory with bulk copies, four (BF16)
// or three (FP32) sub-tiles ahead (one elected producer thread, full/empty
// mbarriers, every wait bounded), for the scenes whose planes allow it, and
// loads the rest directly. The autotuner times the candidate schedules on the
// caller's own prepared batch and returns the fastest.
#include <algorithm>
#include <vector>

#include "nasg_kernels.cuh"

namespace nasg {

struct SceneDev {
  const void* params;
  const void* c0;
  const float* means;
  const float* g_rgb;
  float* rgb;
  float* g_params;
  float* g_c0;
  float* g_means;
  int64_t n;
  int64_t tile_begin;  // first global tile of this scene
  float cam[3];
  int32_t n_lobes;
  int32_t slice_log2;
  int32_t staged;  // parameter spans may be moved by bulk copies (even L, 16-byte aligned planes)
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
  int32_t identity;
  int32_t normalised;
  int32_t exact;
  int* dev_err;
};

template <typename T, int P>
__device__ __forceinline__ void fetch_scene_item(const SceneDev& sc, int64_t prim, int l0, bool valid,
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

// View of one scene as the single-scene argument block (fields eval_item reads).
__device__ __forceinline__ EvalArgs scene_args(const SceneDev& sc, const BatchArgs& b) {
  EvalArgs a;
  a.params = sc.params;
  a.c0 = sc.c0;
  a.means = sc.means;
  a.cam[0] = sc.cam[0];
  a.cam[1] = sc.cam[1];
  a.cam[2] = sc.cam[2];
  a.idx = nullptr;
  a.n_items = sc.n;
  a.n = sc.n;
  a.n_lobes = sc.n_lobes;
  a.slice_log2 = sc.slice_log2;
  a.slice = 1 << sc.slice_log2;
  a.identity = b.identity;
  a.normalised = b.normalised;
  a.exact = b.exact;
  a.accumulate = 0;
  a.g_rgb = sc.g_rgb;
  a.rgb = sc.rgb;
  a.g_params = sc.g_params;
  a.g_c0 = sc.g_c0;
  a.g_means = sc.g_means;
  a.dev_err = b.dev_err;
  return a;
}

// FLAGS: kFlagsDefault (raw activations, approximate normalisation) or
// kFlagsRuntime (modes read from the arguments).
template <int FRAME, typename T, int FLAGS>
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
    const SceneDev& sc = sd[lo];
    const EvalArgs a = scene_args(sc, b);
    const int tp = 256 >> sc.slice_log2;
    const int local = threadIdx.x >> sc.slice_log2;
    const int l0 = 2 * (threadIdx.x & ((1 << sc.slice_log2) - 1));
    const int64_t base = (tile - sc.tile_begin) * int64_t(tp) * b.sub_tiles;
    RawItem<T, P> cur, nxt;
    fetch_scene_item<T, P>(sc, base + local, l0, true, cur);
    for (int j = 0; j < b.sub_tiles; ++j) {
      const int64_t prim = base + int64_t(j) * tp + local;
      fetch_scene_item<T, P>(sc, prim + tp, l0, j + 1 < b.sub_tiles, nxt);
      eval_item<FRAME, T, int64_t, kFwdBwd, false, FLAGS>(a, cur, prim, l0);
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

// Stages in flight per block (f32 parameters take twice the space).
template <typename T>
constexpr int batch_stages() { return sizeof(T) == 2 ? 4 : 3; }
constexpr int kMaxBatchStages = 4;
constexpr uint32_t kUnitEnd = 0xffffffffu;

// Shared-memory metadata of one stage, written by the producer with the unit.
struct StageMeta {
  uint32_t unit;     // global sub-tile index, kUnitEnd past the last
  int32_t scene;     // scene index, -1 for an empty unit
  int32_t staged;    // bit 0: parameter spans in the stage; bit 1: means and upstream gradients too
  int32_t count;     // primitives in the unit
  int64_t p0;        // first primitive of the unit in its scene
};

// Stage layout: P parameter spans of up to 512 lobes, then up to 256 means and
// 256 upstream gradients (a sub-tile holds at most 512 lobes: 256/S primitives x
// L lobes with S >= L/2).
template <typename T, int P>
__host__ __device__ inline uint32_t batch_plane_bytes() { return 512u * uint32_t(sizeof(T)); }
template <typename T, int P>
__host__ __device__ inline uint32_t batch_stage_bytes() {
  return (uint32_t(P) * batch_plane_bytes<T, P>() + 2u * 256u * 12u + 127u) & ~127u;
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
  while (sc_i + 1 < b.n_scenes && sd[sc_i + 1].tile_begin * b.sub_tiles <= u) ++sc_i;
  const SceneDev& sc = sd[sc_i];
  const int64_t tp = 256 >> sc.slice_log2;
  const int64_t p0 = (u - sc.tile_begin * b.sub_tiles) * tp;
  const int64_t count = sc.n - p0 < tp ? sc.n - p0 : tp;
  meta->unit = unit;
  meta->scene = count > 0 ? sc_i : -1;
  meta->count = count > 0 ? int32_t(count) : 0;
  meta->p0 = p0;
  const uint32_t bytes = count > 0 ? uint32_t(count) * uint32_t(sc.n_lobes) * uint32_t(sizeof(T)) : 0u;
  const bool stage_p = count > 0 && (sc.staged & 1) && (bytes % 16u) == 0u;
  const bool stage_m = stage_p && (sc.staged & 2) && (count % 4) == 0;  // 12-byte records: 4 per 16 bytes
  meta->staged = (stage_p ? 1 : 0) | (stage_m ? 2 : 0);
  if (!stage_p) {
    mbar_arrive(bar);
    return false;
  }
  const uint32_t mbytes = uint32_t(count) * 12u;
  mbar_arrive_expect_tx(bar, uint32_t(P) * bytes + (stage_m ? 2u * mbytes : 0u));
  const T* params = static_cast<const T*>(sc.params);
  const int64_t NL = sc.n * sc.n_lobes;
#pragma unroll
  for (int p = 0; p < P; ++p)
    bulk_g2s(st + size_t(p) * batch_plane_bytes<T, P>(), params + p * NL + p0 * sc.n_lobes, bytes, bar);
  if (stage_m) {
    unsigned char* mu = st + size_t(P) * batch_plane_bytes<T, P>();
    bulk_g2s(mu, sc.means + 3 * p0, mbytes, bar);
    bulk_g2s(mu + 256u * 12u, sc.g_rgb + 3 * p0, mbytes, bar);
  }
  return true;
}

template <int FRAME, typename T, int FLAGS>
__global__ void __launch_bounds__(256, 2) batched_staged_kernel(const BatchArgs b) {
  constexpr int P = FrameTraits<FRAME>::P;
  constexpr int NS = batch_stages<T>();
  using W = typename RawWord<T>::type;
  __shared__ SceneDev sd[kMaxScenes];
  __shared__ StageMeta meta[kMaxBatchStages];
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t sbytes = batch_stage_bytes<T, P>();
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * sbytes);
  uint64_t* empty = full + NS;
  {
    const int words = int(b.n_scenes * sizeof(SceneDev) / sizeof(uint32_t));
    const uint32_t* src = reinterpret_cast<const uint32_t*>(b.table);
    uint32_t* dst = reinterpret_cast<uint32_t*>(sd);
    for (int j = threadIdx.x; j < words; j += blockDim.x) dst[j] = src[j];
  }
  const uint32_t n_warps = blockDim.x >> 5;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], n_warps);
    }
    fence_barrier_init();
  }
  __syncthreads();
  // producer state (thread 0): stages whose copies are in flight and the parity of
  // the phase each of them completes, for the drain on error
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
  int cur_scene = -1;
  EvalArgs a{};
  for (uint32_t it = 0;; ++it) {
    if (threadIdx.x == 0 && it >= 1) {
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
    if (threadIdx.x == 0) pending &= ~(1u << s);
    const StageMeta m = meta[s];
    if (m.unit == kUnitEnd) break;  // block-uniform: every warp reads the same stage
    RawItem<T, P> r;
    r.ok = 0;
    int64_t prim = 0;
    int l0 = 0;
    if (m.scene >= 0) {
      const SceneDev& sc = sd[m.scene];
      if (m.scene != cur_scene) {  // block-uniform
        a = scene_args(sc, b);
        cur_scene = m.scene;
      }
      const int local = int(threadIdx.x) >> sc.slice_log2;
      l0 = 2 * (int(threadIdx.x) & ((1 << sc.slice_log2) - 1));
      prim = m.p0 + local;
      if (m.staged & 1) {
        r.ok = local < m.count;
        if (r.ok) {
          r.i = 0;
          const unsigned char* st = smem + s * sbytes;
          if (m.staged & 2) {
            const float* mu = reinterpret_cast<const float*>(st + size_t(P) * batch_plane_bytes<T, P>());
#pragma unroll
            for (int c = 0; c < 3; ++c) r.mu[c] = mu[3 * local + c];
#pragma unroll
            for (int c = 0; c < 3; ++c) r.gc[c] = mu[256 * 3 + 3 * local + c];
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) r.mu[c] = __ldg(sc.means + 3 * prim + c);
#pragma unroll
            for (int c = 0; c < 3; ++c) r.gc[c] = __ldg(sc.g_rgb + 3 * prim + c);
          }
          const T* c0 = static_cast<const T*>(sc.c0);
#pragma unroll
          for (int c = 0; c < 3; ++c) r.c0[c] = load1<T>(c0 + c * sc.n + prim);
          if (l0 < sc.n_lobes) {
#pragma unroll
            for (int p = 0; p < P; ++p)
              r.w[p] = *reinterpret_cast<const W*>(st + size_t(p) * batch_plane_bytes<T, P>() +
                                                   size_t(local * sc.n_lobes + l0) * sizeof(T));
          }
        }
      } else {
        fetch_scene_item<T, P>(sc, prim, l0, true, r);
      }
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
    if (m.scene >= 0) eval_item<FRAME, T, int64_t, kFwdBwd, false, FLAGS>(a, r, prim, l0);
  }
  // on a failed wait, let the copies this block started finish before leaving (bounded)
  if (threadIdx.x == 0 && failed) {
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
  std::vector<SceneDev> tab(n_scenes);
  int64_t tiles = 0, prims = 0, lobes = 0;
  for (int j = 0; j < n_scenes; ++j) {
    const nasg_scene& s = scenes[j];
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
    d.params = s.params;
    d.c0 = s.c0;
    d.means = s.means;
    d.g_rgb = s.g_rgb;
    d.rgb = s.rgb;
    d.g_params = s.g_params;
    d.g_c0 = s.g_c0;
    d.g_means = s.g_means;
    d.n = s.n;
    d.cam[0] = s.cam[0];
    d.cam[1] = s.cam[1];
    d.cam[2] = s.cam[2];
    d.n_lobes = s.n_lobes;
    d.slice_log2 = slice_log2(s.n_lobes);
    d.staged = (s.n_lobes % 2 == 0) && s.params && aligned(s.params, 16) && (s.n * s.n_lobes * es) % 16 == 0
                   ? 1 | (aligned(s.means, 16) && aligned(s.g_rgb, 16) ? 2 : 0)
                   : 0;
    d.tile_begin = tiles;
    const int64_t tile_prims = int64_t(256 >> d.slice_log2) * sub_tiles;
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
  plan->total_tiles = tiles;
  plan->total_prims = prims;
  plan->total_lobes = lobes;
  plan->workspace = workspace;
  return NASG_OK;
}

namespace nasg {
template <int FRAME, typename T>
static nasg_status launch_batched(const BatchArgs& b, int blocks_per_sm, bool staged, cudaStream_t s) {
  const bool dflt = b.identity == 0 && b.normalised != 0 && b.exact == 0;
  if (staged) {
    constexpr int P = FrameTraits<FRAME>::P;
    auto k = dflt ? batched_staged_kernel<FRAME, T, kFlagsDefault> : batched_staged_kernel<FRAME, T, kFlagsRuntime>;
    constexpr int NS = batch_stages<T>();
    const size_t smem = size_t(NS) * batch_stage_bytes<T, P>() + 2 * NS * sizeof(uint64_t);
    static size_t configured[2] = {0, 0};  // per instantiation pair (default, run-time flags)
    size_t& cfg = configured[dflt ? 0 : 1];
    if (smem > cfg) {
      if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        return check_launch();
      cfg = smem;
    }
    int fit = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k, 256, smem) != cudaSuccess || fit < 1) fit = 1;
    const int per_sm = blocks_per_sm > 0 && blocks_per_sm < fit ? blocks_per_sm : fit;
    int64_t grid = int64_t(sm_count()) * per_sm;
    const int64_t units = b.total_tiles * b.sub_tiles;
    if (grid > units) grid = units;
    if (grid < 1) return NASG_OK;
    k<<<unsigned(grid), 256, smem, s>>>(b);
    return check_launch();
  }
  auto k = dflt ? batched_kernel<FRAME, T, kFlagsDefault> : batched_kernel<FRAME, T, kFlagsRuntime>;
  int fit = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k, 256, 0) != cudaSuccess || fit < 1) fit = 1;
  const int per_sm = blocks_per_sm > 0 && blocks_per_sm < fit ? blocks_per_sm : fit;
  int64_t grid = int64_t(sm_count()) * per_sm;
  if (grid > b.total_tiles) grid = b.total_tiles;
  if (grid < 1) return NASG_OK;
  k<<<unsigned(grid), 256, 0, s>>>(b);
  return check_launch();
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
  unsigned char* ws = static_cast<unsigned char*>(plan->workspace);
  cudaStream_t st = as_stream(stream);
  BatchArgs b{};
  b.table = reinterpret_cast<const SceneDev*>(ws + kBatchHeader);
  b.counter = reinterpret_cast<uint32_t*>(ws);
  b.n_scenes = plan->n_scenes;
  b.sub_tiles = plan->sub_tiles;
  b.total_tiles = plan->total_tiles;
  b.dynamic = dynamic;
  b.identity = plan->act_mode == NASG_ACT_IDENTITY;
  b.normalised = plan->norm_mode != NASG_NORM_NONE;
  b.exact = plan->norm_mode == NASG_NORM_EXACT;
  b.dev_err = device_error_word();
  if (dynamic && cudaMemsetAsync(b.counter, 0, sizeof(uint32_t), st) != cudaSuccess) return check_launch();
  const bool quat = plan->frame_mode == NASG_FRAME_QUAT;
  const bool bf16 = plan->param_dtype == NASG_DTYPE_BF16;
  if (quat) {
    return bf16 ? launch_batched<NASG_FRAME_QUAT, __nv_bfloat16>(b, bps, staged, st)
                : launch_batched<NASG_FRAME_QUAT, float>(b, bps, staged, st);
  }
  return bf16 ? launch_batched<NASG_FRAME_COS, __nv_bfloat16>(b, bps, staged, st)
              : launch_batched<NASG_FRAME_COS, float>(b, bps, staged, st);
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
        for (int r = 0; r < reps; ++r) nasgabor_batched_run(&pl, &t, stream);
        cudaEventRecord(e1, st);
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
