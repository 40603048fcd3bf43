// Fused forward + backward + Adam training step of the NASGabor appearance
// model (nasgabor_fused_step) and the frustum visibility compaction that
// produces its index list (nasg_frustum_compact).
//
// Step: for every listed primitive, the lobes are evaluated at the stored
// parameter values (RNE bfloat16 of the FP32 master when desc->param_dtype is
// BF16), the Supp. F gradients for the upstream dLoss/dRGB are formed in
// registers (never written to memory), and Adam (bias-corrected, in
// torch.optim.Adam's operation order) updates master, m and v in place and
// writes the BF16 copy. Primitives not listed are not touched. The upstream
// gradient is either given, or (loss mode MSE) formed in the kernel from the
// primitive's colour and a target colour: the loss is the mean over the listed
// primitives and the three channels of (c - target)^2, so dLoss/dc =
// 2 (c - target) / (3 n_listed), which needs the primitive's whole colour before
// the backward starts (the lanes' lobe partials wait in registers across the
// slice reduction). Mapping and numerics are those of the evaluation kernels
// (nasg_kernels.cuh): a lane holds two lobes in packed FP32x2 arithmetic and a
// slice of lanes covers a primitive.
//
// Compaction: an ordered (deterministic, ascending) list of the primitives
// whose centre is inside a pinhole frustum, in three launches: per-chunk
// counts (and a visibility byte per primitive), one-block exclusive scan of the
// counts (also the total), and the ordered scatter.
#include <cmath>
#include <mutex>

#include "nasg_kernels.cuh"

namespace nasg {

struct StepArgs {
  EvalArgs e;            // params = master, c0 = c0 master, g_rgb, rgb (nullable), g_means (nullable)
  float* m;              // [P][N*L]
  float* v;              // [P][N*L]
  uint16_t* pbf;         // [P][N*L] bf16 copy, nullable
  float* c0m;            // [3][N]
  float* c0v;            // [3][N]
  uint16_t* c0bf;        // [3][N] bf16 copy, nullable
  const int32_t* n_dev;  // device item count (min with e.n_items), nullable
  float b1, b2, omb1, omb2, step_size, inv_sqrt_bc2, eps;
  int32_t quantize;      // evaluate at RNE_bf16(master)
};

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float bf16_rne(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

// Per-thread 8-byte asynchronous global -> shared copy (cp.async: no register
// staging; source and destination 8-byte aligned), and the wait for all of the
// thread's own copies. Used for the Adam state of a lane's two lobes, issued
// before the lobe math so that its latency overlaps the arithmetic.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One bias-corrected Adam update: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
// th <- th - (lr/bc1) m / (sqrt(v)/sqrt(bc2) + eps).
__device__ __forceinline__ void adam(const StepArgs& s, float g, float& th, float& m, float& v) {
  m = fmaf(s.b1, m, s.omb1 * g);
  v = fmaf(s.b2, v, s.omb2 * (g * g));
  const float den = fmaf(sqrt_approx(v), s.inv_sqrt_bc2, s.eps);
  th = fmaf(-s.step_size, m * rcpa(den), th);
}

// Phase one of a step item: the lobe math. The lane's P gradient pairs are
// parked in its own shared-memory slot (gslot[p * 256]) rather than kept in
// registers, so that phase two starts with a fresh register budget and can
// issue all of its moment and master loads at once. Also does the
// per-primitive work (colour, dLoss/dmu, c0 Adam). LOSS: cur.gc holds the
// target colour and gscale = 2 / (3 n_listed); the upstream gradient is
// gscale (colour - target). Returns whether the lane holds lobes to update.
template <int FRAME, typename IDX, bool EVEN, bool LOSS>
__device__ __forceinline__ bool step_phase1(const StepArgs& s, const RawItem<float, FrameTraits<FRAME>::P>& cur,
                                            IDX i, int l0, float gscale, float2* gslot) {
  constexpr int P = FrameTraits<FRAME>::P;
  const EvalArgs& a = s.e;
  const IDX n = IDX(a.n);
  const IDX L = IDX(a.n_lobes);
  const bool ok = cur.ok != 0;
  const bool quant = s.quantize != 0;
  bool mine = false;
  float rgb[3] = {0.f, 0.f, 0.f};
  float gd[3] = {0.f, 0.f, 0.f};
  float d[3] = {0.f, 0.f, 1.f};
  float gc[3] = {cur.gc[0], cur.gc[1], cur.gc[2]};  // LOSS: the target until the residual is formed
  float inv_dist = 0.f;
  bool second = true;
  P2 dv[3];
  LobeEval<FRAME, P2> ev;
  if (ok) {
    inv_dist = view_dir_rn(cur.mu, a.cam, d);
    if (IDX(l0) < L) {
      mine = true;
      second = EVEN || (IDX(l0) + 1 < L);
      P2 pv[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const float2 w = cur.w[p];
        pv[p] = quant ? p2(bf16_rne(w.x), bf16_rne(w.y)) : p2(w.x, w.y);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) dv[c] = p2(d[c]);
      if (LOSS) {
        lobe_eval<FRAME, true>(pv, dv, a.identity != 0, a.normalised != 0, a.exact != 0, ev);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const P2 t = ev.act.w[c] * ev.G;
          rgb[c] = t.v.x + (second ? t.v.y : 0.f);
        }
      } else {
        const P2 gcv[3] = {p2(gc[0]), p2(gc[1]), p2(gc[2])};
        P2 rgbv[3] = {p2(0.f), p2(0.f), p2(0.f)};
        P2 gdv[3] = {p2(0.f), p2(0.f), p2(0.f)};
        P2 gp[P];
        lobe_step<FRAME, true, true>(pv, dv, gcv, a.identity != 0, a.normalised != 0, a.exact != 0, rgbv, gdv, gp);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          rgb[c] = rgbv[c].v.x + (second ? rgbv[c].v.y : 0.f);
          gd[c] = gdv[c].v.x + (second ? gdv[c].v.y : 0.f);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) gslot[p * 256] = gp[p].v;
      }
    }
  }
  float c0e[3];  // diffuse colour as evaluated (the BF16 value when quantising)
#pragma unroll
  for (int c = 0; c < 3; ++c) c0e[c] = quant ? bf16_rne(cur.c0[c]) : cur.c0[c];
  if (LOSS) {
    // the primitive's colour in every lane of the slice, then the residual
    for (int o = a.slice >> 1; o >= 1; o >>= 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) rgb[c] += __shfl_xor_sync(0xffffffffu, rgb[c], o);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) gc[c] = gscale * ((rgb[c] + c0e[c]) - gc[c]);
    if (mine) {
      const P2 gcv[3] = {p2(gc[0]), p2(gc[1]), p2(gc[2])};
      P2 gdv[3] = {p2(0.f), p2(0.f), p2(0.f)};
      P2 gp[P];
      lobe_grad<FRAME>(ev, dv, gcv, gdv, gp);
#pragma unroll
      for (int c = 0; c < 3; ++c) gd[c] = gdv[c].v.x + (second ? gdv[c].v.y : 0.f);
#pragma unroll
      for (int p = 0; p < P; ++p) gslot[p * 256] = gp[p].v;
    }
    for (int o = a.slice >> 1; o >= 1; o >>= 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) gd[c] += __shfl_xor_sync(0xffffffffu, gd[c], o);
    }
  } else {
    for (int o = a.slice >> 1; o >= 1; o >>= 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        rgb[c] += __shfl_xor_sync(0xffffffffu, rgb[c], o);
        gd[c] += __shfl_xor_sync(0xffffffffu, gd[c], o);
      }
    }
  }
  if (ok) {
    const float dot = dot3_rn(gd, d);
    for (int c = l0 >> 1; c < 3; c += a.slice) {
      float th = pick3(cur.c0, c);
      if (a.rgb) a.rgb[3 * i + c] = pick3(rgb, c) + pick3(c0e, c);
      if (a.g_means) a.g_means[3 * i + c] = mean_grad_rn(pick3(gd, c), dot, pick3(d, c), inv_dist);
      const IDX o = IDX(c) * n + i;
      float mm = s.c0m[o], vv = s.c0v[o];
      adam(s, pick3(gc, c), th, mm, vv);
      float* c0master = static_cast<float*>(const_cast<void*>(a.c0));
      c0master[o] = th;
      s.c0m[o] = mm;
      s.c0v[o] = vv;
      if (s.c0bf) s.c0bf[o] = bf16_bits(th);
    }
  }
  return mine;
}

// Phase two: Adam on the lane's two lobes for every plane. EVEN: master, m and v
// were copied into the lane's shared-memory slots (tslot, mslot, vslot: plane p
// at [p * 256]) while phase one ran. Otherwise in batches of planes: all loads of
// a batch first (master, m, v), then the updates and stores.
template <int P, typename IDX, bool EVEN>
__device__ __forceinline__ void step_phase2(const StepArgs& s, IDX i, int l0, const float2* gslot,
                                            const float2* tslot, const float2* mslot, const float2* vslot) {
  constexpr int kBatch = EVEN ? P : (P + 1) / 2;
  const EvalArgs& a = s.e;
  const IDX n = IDX(a.n);
  const IDX L = IDX(a.n_lobes);
  const IDX NL = n * L;
  const IDX off0 = i * L + IDX(l0);
  const bool second = EVEN || (IDX(l0) + 1 < L);
  float* master = static_cast<float*>(const_cast<void*>(a.params));
#pragma unroll
  for (int p0 = 0; p0 < P; p0 += kBatch) {
    float2 th[kBatch], mm[kBatch], vv[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      if (p0 + j >= P) break;
      const IDX off = off0 + IDX(p0 + j) * NL;
      if (EVEN) {
        th[j] = tslot[(p0 + j) * 256];
        mm[j] = mslot[(p0 + j) * 256];
        vv[j] = vslot[(p0 + j) * 256];
      } else {
        th[j] = make_float2(master[off], second ? master[off + 1] : 0.f);
        mm[j] = make_float2(s.m[off], second ? s.m[off + 1] : 0.f);
        vv[j] = make_float2(s.v[off], second ? s.v[off + 1] : 0.f);
      }
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      if (p0 + j >= P) break;
      const float2 g = gslot[(p0 + j) * 256];
      adam(s, g.x, th[j].x, mm[j].x, vv[j].x);
      adam(s, g.y, th[j].y, mm[j].y, vv[j].y);
      const IDX off = off0 + IDX(p0 + j) * NL;
      if (EVEN) {
        *reinterpret_cast<float2*>(master + off) = th[j];
        *reinterpret_cast<float2*>(s.m + off) = mm[j];
        *reinterpret_cast<float2*>(s.v + off) = vv[j];
        if (s.pbf) {
          const uint32_t w2 = uint32_t(bf16_bits(th[j].x)) | (uint32_t(bf16_bits(th[j].y)) << 16);
          *reinterpret_cast<uint32_t*>(s.pbf + off) = w2;
        }
      } else {
        master[off] = th[j].x; s.m[off] = mm[j].x; s.v[off] = vv[j].x;
        if (s.pbf) s.pbf[off] = bf16_bits(th[j].x);
        if (second) {
          master[off + 1] = th[j].y; s.m[off + 1] = mm[j].y; s.v[off + 1] = vv[j].y;
          if (s.pbf) s.pbf[off + 1] = bf16_bits(th[j].y);
        }
      }
    }
  }
}

// Shared memory of the step kernel: per thread, P gradient pairs and (EVEN) the
// P master, m and v pairs of its two lobes, each plane-major over the block's
// 256 threads (no sharing between threads, no barrier).
template <int P, bool EVEN>
constexpr size_t step_smem_bytes() { return size_t(EVEN ? 4 : 1) * P * 256 * sizeof(float2); }

template <int FRAME, typename IDX, bool EVEN, bool LOSS>
__global__ void __launch_bounds__(256, 2) step_kernel(const StepArgs s) {
  constexpr int P = FrameTraits<FRAME>::P;
  extern __shared__ __align__(16) float2 step_smem[];
  const EvalArgs& a = s.e;
  int64_t items = a.n_items;
  if (s.n_dev) {
    const int64_t dn = int64_t(__ldg(s.n_dev));
    items = dn < 0 ? 0 : (dn < items ? dn : items);
  }
  const int l0 = 2 * (threadIdx.x & (a.slice - 1));
  const IDX total = IDX(items) << a.slice_log2;
  const IDX stride = IDX(gridDim.x) * blockDim.x;
  const float gscale = LOSS && items > 0 ? 2.f / (3.f * float(items)) : 0.f;  // d mean / d colour
  float2* gslot = step_smem + threadIdx.x;
  float2* tslot = gslot + P * 256;
  float2* mslot = tslot + P * 256;
  float2* vslot = mslot + P * 256;
  const IDX L = IDX(a.n_lobes);
  const IDX NL = IDX(a.n) * L;
  const float* master = static_cast<const float*>(a.params);
  // block-uniform loop: every lane of a warp reaches the shuffles in phase one
  for (IDX t0 = IDX(blockIdx.x) * blockDim.x; t0 < total; t0 += stride) {
    RawItem<float, P> cur;
    IDX i = 0;
    fetch_item<float, P, IDX, EVEN, true, true>(a, total, t0 + threadIdx.x, l0, cur, i);
    if (EVEN && cur.ok && IDX(l0) < L) {
      IDX off = i * L + IDX(l0);
#pragma unroll
      for (int p = 0; p < P; ++p, off += NL) {
        cp_async8(tslot + p * 256, master + off);
        cp_async8(mslot + p * 256, s.m + off);
        cp_async8(vslot + p * 256, s.v + off);
      }
    }
    const bool mine = step_phase1<FRAME, IDX, EVEN, LOSS>(s, cur, i, l0, gscale, gslot);
    if (EVEN) cp_async_wait_all();
    if (mine) step_phase2<P, IDX, EVEN>(s, i, l0, gslot, tslot, mslot, vslot);
  }
}

template <int FRAME, typename IDX, bool EVEN, bool LOSS>
static nasg_status launch_step_k(const StepArgs& s, cudaStream_t st) {
  constexpr int P = FrameTraits<FRAME>::P;
  constexpr size_t smem = step_smem_bytes<P, EVEN>();
  auto k = step_kernel<FRAME, IDX, EVEN, LOSS>;
  if (const nasg_status e = ensure_smem_limit(reinterpret_cast<const void*>(k), smem); e != NASG_OK) return e;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
  const int64_t threads = s.e.n_items << s.e.slice_log2;
  const unsigned need = grid_for(threads, 256);
  const unsigned cap = unsigned(sm_count() * per_sm);
  k<<<need < cap ? need : cap, 256, smem, st>>>(s);
  return check_launch();
}

template <int FRAME, typename IDX>
static nasg_status launch_step_idx(const StepArgs& s, bool even, bool loss, cudaStream_t st) {
  if (loss) return even ? launch_step_k<FRAME, IDX, true, true>(s, st) : launch_step_k<FRAME, IDX, false, true>(s, st);
  return even ? launch_step_k<FRAME, IDX, true, false>(s, st) : launch_step_k<FRAME, IDX, false, false>(s, st);
}

// ---------------------------------------------------------------------------
// Frustum compaction
// ---------------------------------------------------------------------------

constexpr int kCompactBlock = 256;
constexpr int kCompactChunk = 4096;  // primitives per block (16 rounds of 256)

struct FrustumArgs {
  const float* means;
  int64_t n;
  float r[9];  // world -> camera rows: right, up, forward
  float c[3];  // camera centre
  float t;     // tan(fov/2)
  float near_z;
};

// Visibility of one centre with explicitly rounded operations, so that every
// launch makes the identical decision.
__device__ __forceinline__ bool in_frustum(const FrustumArgs& f, int64_t i) {
  const float x = __fsub_rn(f.means[3 * i + 0], f.c[0]);
  const float y = __fsub_rn(f.means[3 * i + 1], f.c[1]);
  const float z = __fsub_rn(f.means[3 * i + 2], f.c[2]);
  const float px = __fmaf_rn(f.r[0], x, __fmaf_rn(f.r[1], y, __fmul_rn(f.r[2], z)));
  const float py = __fmaf_rn(f.r[3], x, __fmaf_rn(f.r[4], y, __fmul_rn(f.r[5], z)));
  const float pz = __fmaf_rn(f.r[6], x, __fmaf_rn(f.r[7], y, __fmul_rn(f.r[8], z)));
  const float lim = __fmul_rn(f.t, pz);
  return pz > f.near_z && fabsf(px) <= lim && fabsf(py) <= lim;
}

__global__ void __launch_bounds__(kCompactBlock) frustum_count_kernel(FrustumArgs f, uint8_t* flags,
                                                                      int32_t* counts) {
  const int64_t base = int64_t(blockIdx.x) * kCompactChunk;
  int local = 0;
  for (int r = 0; r < kCompactChunk / kCompactBlock; ++r) {
    const int64_t i = base + r * kCompactBlock + threadIdx.x;
    const bool v = i < f.n && in_frustum(f, i);
    if (i < f.n) flags[i] = v ? 1 : 0;
    local += __syncthreads_count(v);
  }
  if (threadIdx.x == 0) counts[blockIdx.x] = local;
}

// One block: exclusive prefix over counts[0..nb) -> offsets, total -> *n_visible.
__global__ void __launch_bounds__(1024) frustum_scan_kernel(const int32_t* counts, int32_t* offsets, int32_t nb,
                                                            int32_t* n_visible) {
  __shared__ int32_t part[1024];
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  int32_t sum = 0;
  for (int j = 0; j < per; ++j)
    if (b0 + j < nb) sum += counts[b0 + j];
  part[threadIdx.x] = sum;
  __syncthreads();
  // Hillis-Steele inclusive scan of the per-thread sums
  for (int o = 1; o < int(blockDim.x); o <<= 1) {
    const int32_t add = threadIdx.x >= unsigned(o) ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  int32_t run = part[threadIdx.x] - sum;  // exclusive
  for (int j = 0; j < per; ++j) {
    if (b0 + j < nb) {
      offsets[b0 + j] = run;
      run += counts[b0 + j];
    }
  }
  if (threadIdx.x == blockDim.x - 1) *n_visible = part[threadIdx.x];
}

__global__ void __launch_bounds__(kCompactBlock) frustum_scatter_kernel(int64_t n, const uint8_t* flags,
                                                                        const int32_t* offsets, int32_t* idx) {
  __shared__ int32_t warp_tot[kCompactBlock / 32];
  const int64_t base = int64_t(blockIdx.x) * kCompactChunk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t run = offsets[blockIdx.x];
  for (int r = 0; r < kCompactChunk / kCompactBlock; ++r) {
    const int64_t i = base + r * kCompactBlock + threadIdx.x;
    const bool v = i < n && flags[i] != 0;
    const unsigned bal = __ballot_sync(0xffffffffu, v);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int32_t before = 0, round = 0;
#pragma unroll
    for (int w = 0; w < kCompactBlock / 32; ++w) {
      const int32_t t = warp_tot[w];
      before += w < warp ? t : 0;
      round += t;
    }
    if (v) idx[run + before + __popc(bal & ((1u << lane) - 1u))] = int32_t(i);
    run += round;
    __syncthreads();
  }
}

static int64_t compact_blocks(int64_t n) { return (n + kCompactChunk - 1) / kCompactChunk; }

}  // namespace nasg

using namespace nasg;

extern "C" size_t nasg_frustum_workspace_bytes(int64_t n) {
  if (n < 0) return 0;
  const int64_t nb = compact_blocks(n);
  return size_t((n + 15) / 16 * 16) + size_t(2 * nb) * sizeof(int32_t);
}

extern "C" nasg_status nasg_frustum_compact(int64_t n, const float* means, const float* rot, const float* center,
                                            float tan_half_fov, float near_z, int32_t* idx, int32_t* n_visible,
                                            void* workspace, size_t workspace_bytes, void* stream) {
  if (n < 0 || n >= (int64_t(1) << 31)) return NASG_ERR_RANGE;
  if (!rot || !center || !n_visible) return NASG_ERR_NULL;
  if (!(tan_half_fov > 0.f)) return NASG_ERR_RANGE;
  cudaStream_t s = as_stream(stream);
  if (n == 0) {
    if (cudaMemsetAsync(n_visible, 0, sizeof(int32_t), s) != cudaSuccess) return check_launch();
    return NASG_OK;
  }
  if (!means || !idx || !workspace) return NASG_ERR_NULL;
  if (!aligned(means, 4) || !aligned(idx, 4) || !aligned(n_visible, 4) || !aligned(workspace, 16))
    return NASG_ERR_ALIGN;
  if (workspace_bytes < nasg_frustum_workspace_bytes(n)) return NASG_ERR_RANGE;
  const int64_t nb = compact_blocks(n);
  uint8_t* flags = static_cast<uint8_t*>(workspace);
  int32_t* counts = reinterpret_cast<int32_t*>(flags + (n + 15) / 16 * 16);
  int32_t* offsets = counts + nb;
  FrustumArgs f{};
  f.means = means;
  f.n = n;
  for (int j = 0; j < 9; ++j) f.r[j] = rot[j];
  for (int j = 0; j < 3; ++j) f.c[j] = center[j];
  f.t = tan_half_fov;
  f.near_z = near_z;
  frustum_count_kernel<<<unsigned(nb), kCompactBlock, 0, s>>>(f, flags, counts);
  frustum_scan_kernel<<<1, 1024, 0, s>>>(counts, offsets, int32_t(nb), n_visible);
  frustum_scatter_kernel<<<unsigned(nb), kCompactBlock, 0, s>>>(n, flags, offsets, idx);
  return check_launch();
}

extern "C" nasg_status nasgabor_fused_step(const nasg_desc* desc, const nasg_train_state* st, const float* means,
                                           const float* cam, const int32_t* idx, int64_t n_idx,
                                           const int32_t* n_idx_device, const float* g_rgb, int32_t loss_mode,
                                           const nasg_adam_hparams* hp, float* rgb, float* g_means, void* stream) {
  nasg_status e = check_desc(desc);
  if (e != NASG_OK) return e;
  if (desc->lobe_family != NASG_FAMILY_NASGABOR) return NASG_ERR_UNSUPPORTED;
  if (desc->accumulate != 0) return NASG_ERR_RANGE;
  if (loss_mode != NASG_LOSS_GIVEN && loss_mode != NASG_LOSS_MSE) return NASG_ERR_RANGE;
  if (!st || !hp || !cam) return NASG_ERR_NULL;
  if (idx && n_idx < 0) return NASG_ERR_RANGE;
  if (hp->step < 1 || !(hp->lr >= 0.f) || !(hp->beta1 >= 0.f && hp->beta1 < 1.f) ||
      !(hp->beta2 >= 0.f && hp->beta2 < 1.f) || !(hp->eps > 0.f))
    return NASG_ERR_RANGE;
  if (desc->n == 0 || (idx && n_idx == 0)) return NASG_OK;
  if (!st->master || !st->m || !st->v || !st->c0_master || !st->c0_m || !st->c0_v || !means || !g_rgb)
    return NASG_ERR_NULL;
  const void* f32[] = {st->master, st->m, st->v, st->c0_master, st->c0_m, st->c0_v, means, g_rgb, rgb, g_means};
  for (const void* p : f32)
    if (p && !aligned(p, 4)) return NASG_ERR_ALIGN;
  if ((st->params_bf16 && !aligned(st->params_bf16, 2)) || (st->c0_bf16 && !aligned(st->c0_bf16, 2)) ||
      (idx && !aligned(idx, 4)) || (n_idx_device && !aligned(n_idx_device, 4)))
    return NASG_ERR_ALIGN;
  StepArgs s{};
  EvalArgs& a = s.e;
  a.params = st->master;
  a.c0 = st->c0_master;
  a.means = means;
  a.cam[0] = cam[0];
  a.cam[1] = cam[1];
  a.cam[2] = cam[2];
  a.idx = idx;
  a.n_items = idx ? n_idx : desc->n;
  a.n = desc->n;
  a.n_lobes = desc->n_lobes;
  a.slice_log2 = slice_log2(desc->n_lobes);
  a.slice = 1 << a.slice_log2;
  a.identity = desc->act_mode == NASG_ACT_IDENTITY;
  a.normalised = desc->norm_mode != NASG_NORM_NONE;
  a.exact = desc->norm_mode == NASG_NORM_EXACT;
  a.g_rgb = g_rgb;
  a.rgb = rgb;
  a.g_means = g_means;
  a.dev_err = device_error_word();
  s.m = st->m;
  s.v = st->v;
  s.pbf = static_cast<uint16_t*>(st->params_bf16);
  s.c0m = st->c0_m;
  s.c0v = st->c0_v;
  s.c0bf = static_cast<uint16_t*>(st->c0_bf16);
  s.n_dev = n_idx_device;
  const double b1 = hp->beta1, b2 = hp->beta2;
  const double bc1 = 1.0 - std::pow(b1, double(hp->step));
  const double bc2 = 1.0 - std::pow(b2, double(hp->step));
  s.b1 = float(b1);
  s.b2 = float(b2);
  s.omb1 = float(1.0 - b1);
  s.omb2 = float(1.0 - b2);
  s.step_size = float(double(hp->lr) / bc1);
  s.inv_sqrt_bc2 = float(1.0 / std::sqrt(bc2));
  s.eps = hp->eps;
  s.quantize = desc->param_dtype == NASG_DTYPE_BF16;
  const bool even = desc->n_lobes % 2 == 0 && aligned(st->master, 8) && aligned(st->m, 8) && aligned(st->v, 8) &&
                    (!st->params_bf16 || aligned(st->params_bf16, 4));
  const int64_t NL = desc->n * desc->n_lobes;
  const int64_t lim = int64_t(1) << 31;
  const bool idx32 = NL * nasg_lobe_planes(desc->frame_mode) < lim && 3 * desc->n < lim &&
                     2 * (a.n_items << a.slice_log2) + (int64_t(1) << 24) < lim;
  cudaStream_t cs = as_stream(stream);
  const bool loss = loss_mode == NASG_LOSS_MSE;
  if (desc->frame_mode == NASG_FRAME_QUAT) {
    return idx32 ? launch_step_idx<NASG_FRAME_QUAT, uint32_t>(s, even, loss, cs)
                 : launch_step_idx<NASG_FRAME_QUAT, uint64_t>(s, even, loss, cs);
  }
  return idx32 ? launch_step_idx<NASG_FRAME_COS, uint32_t>(s, even, loss, cs)
               : launch_step_idx<NASG_FRAME_COS, uint64_t>(s, even, loss, cs);
}

// ---------------------------------------------------------------------------
// BF16 copies of a training state
// ---------------------------------------------------------------------------
namespace nasg {

// dst[j] = RNE_bf16(src[j]), eight elements per thread where both arrays allow
// 16-byte (src) and 16-byte (dst, eight bf16) accesses, single elements otherwise.
__global__ void __launch_bounds__(256) round_bf16_kernel(const float* __restrict__ src, uint16_t* __restrict__ dst,
                                                         int64_t n, int vec) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (vec) {
    const int64_t n8 = n / 8;
    for (; j < n8; j += stride) {
      const float4 a = reinterpret_cast<const float4*>(src)[2 * j];
      const float4 b = reinterpret_cast<const float4*>(src)[2 * j + 1];
      uint4 w;
      w.x = uint32_t(bf16_bits(a.x)) | (uint32_t(bf16_bits(a.y)) << 16);
      w.y = uint32_t(bf16_bits(a.z)) | (uint32_t(bf16_bits(a.w)) << 16);
      w.z = uint32_t(bf16_bits(b.x)) | (uint32_t(bf16_bits(b.y)) << 16);
      w.w = uint32_t(bf16_bits(b.z)) | (uint32_t(bf16_bits(b.w)) << 16);
      reinterpret_cast<uint4*>(dst)[j] = w;
    }
    j = n8 * 8 + (int64_t(blockIdx.x) * blockDim.x + threadIdx.x);
  }
  for (; j < n; j += stride) dst[j] = bf16_bits(src[j]);
}

static nasg_status round_bf16(const float* src, void* dst, int64_t n, cudaStream_t s) {
  if (n == 0 || !dst) return NASG_OK;
  const int vec = aligned(src, 16) && aligned(dst, 16);
  const int64_t work = vec ? n / 8 + 1 : n;
  const unsigned grid = grid_for(work, 256);
  const unsigned cap = unsigned(sm_count()) * 8u;
  round_bf16_kernel<<<grid < cap ? grid : cap, 256, 0, s>>>(src, static_cast<uint16_t*>(dst), n, vec);
  return check_launch();
}

}  // namespace nasg

extern "C" nasg_status nasg_train_state_refresh_bf16(const nasg_desc* desc, const nasg_train_state* st,
                                                     void* stream) {
  nasg_status e = check_desc(desc);
  if (e != NASG_OK) return e;
  if (!st) return NASG_ERR_NULL;
  const int P = nasg_param_planes(desc->frame_mode, desc->lobe_family);
  if (P < 0) return NASG_ERR_UNSUPPORTED;
  if (desc->n == 0) return NASG_OK;
  if ((st->params_bf16 && !st->master) || (st->c0_bf16 && !st->c0_master)) return NASG_ERR_NULL;
  if ((st->master && !aligned(st->master, 4)) || (st->c0_master && !aligned(st->c0_master, 4)) ||
      (st->params_bf16 && !aligned(st->params_bf16, 2)) || (st->c0_bf16 && !aligned(st->c0_bf16, 2)))
    return NASG_ERR_ALIGN;
  cudaStream_t s = as_stream(stream);
  e = round_bf16(st->master, st->params_bf16, int64_t(P) * desc->n * desc->n_lobes, s);
  if (e != NASG_OK) return e;
  return round_bf16(st->c0_master, st->c0_bf16, 3 * desc->n, s);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the frustum compaction
// ---------------------------------------------------------------------------
// Some callers cannot allocate device memory where they need the visible list:
// a renderer plugged into a host application that owns every device allocation
// through its own pool and forbids others, or a per-frame loop with a fixed
// memory budget where a cudaMalloc would synchronise the device and stall the
// frame. For them, nasg_frustum_compact_noalloc keeps its scratch (one
// visibility byte per primitive, per-chunk counts and offsets) in a fixed
// array of this library's device memory instead of a caller-provided
// workspace. The array is sized for NASG_NOALLOC_MAX_PRIMS primitives and is
// held by every GPU that loads the library until the process exits.
namespace nasg {

constexpr int64_t kNoAllocMaxPrims = NASG_NOALLOC_MAX_PRIMS;
constexpr int64_t kNoAllocMaxChunks = (kNoAllocMaxPrims + kCompactChunk - 1) / kCompactChunk;
constexpr size_t kNoAllocScratchBytes =
    size_t((kNoAllocMaxPrims + 15) / 16 * 16) + size_t(2 * kNoAllocMaxChunks) * sizeof(int32_t);

static __device__ __align__(256) unsigned char g_compact_scratch[kNoAllocScratchBytes];

// Device address of g_compact_scratch on the current device. In host code the
// array's name only stands for the symbol, so the address is looked up once per
// device (with that device current) and cached.
static unsigned char* noalloc_scratch() {
  static std::mutex mu;
  static unsigned char* cached[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!cached[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_compact_scratch);
    if (e != cudaSuccess) {
      record_cuda_error(e);
      return nullptr;
    }
    cached[dev] = static_cast<unsigned char*>(p);
  }
  return cached[dev];
}

}  // namespace nasg

extern "C" nasg_status nasg_frustum_compact_noalloc(int64_t n, const float* means, const float* rot,
                                                    const float* center, float tan_half_fov, float near_z,
                                                    int32_t* idx, int32_t* n_visible, void* stream) {
  if (n < 0) return NASG_ERR_RANGE;
  if (n > kNoAllocMaxPrims) return NASG_ERR_CAPACITY;
  if (!rot || !center || !n_visible) return NASG_ERR_NULL;
  if (!(tan_half_fov > 0.f)) return NASG_ERR_RANGE;
  cudaStream_t s = as_stream(stream);
  if (n == 0) {
    if (cudaMemsetAsync(n_visible, 0, sizeof(int32_t), s) != cudaSuccess) return check_launch();
    return NASG_OK;
  }
  if (!means || !idx) return NASG_ERR_NULL;
  if (!aligned(means, 4) || !aligned(idx, 4) || !aligned(n_visible, 4)) return NASG_ERR_ALIGN;
  unsigned char* ws = noalloc_scratch();
  if (!ws) return NASG_ERR_CUDA;
  // Every byte the kernels read is written earlier in the same call (flags for
  // i < n, counts and offsets for the n's chunks), so nothing needs clearing.
  const int64_t nb = compact_blocks(n);
  uint8_t* flags = ws;
  int32_t* counts = reinterpret_cast<int32_t*>(ws + (n + 15) / 16 * 16);
  int32_t* offsets = counts + nb;
  FrustumArgs f{};
  f.means = means;
  f.n = n;
  for (int j = 0; j < 9; ++j) f.r[j] = rot[j];
  for (int j = 0; j < 3; ++j) f.c[j] = center[j];
  f.t = tan_half_fov;
  f.near_z = near_z;
  frustum_count_kernel<<<unsigned(nb), kCompactBlock, 0, s>>>(f, flags, counts);
  frustum_scan_kernel<<<1, 1024, 0, s>>>(counts, offsets, int32_t(nb), n_visible);
  frustum_scatter_kernel<<<unsigned(nb), kCompactBlock, 0, s>>>(n, flags, offsets, idx);
  return check_launch();
}
