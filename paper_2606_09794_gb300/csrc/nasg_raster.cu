// Front-to-back alpha compositing of the primitives (the consumer of the
// per-primitive colours) and its backward to the colours and opacities:
// nasg_raster_forward / nasg_raster_backward.
//
// Sec. 3.1: C(r) = sum_i T_i alpha_i c_i, alpha_i = sigma_i rho_i,
// T_i = prod_{j<i} (1 - alpha_j), with rho_i the primitive's Gaussian kernel
// projected onto the image plane. Rules (the compositing conventions of the
// Gaussian-splatting rasterizer the paper builds on):
//   camera      p = R (mu - centre), rows (right, up, forward); x = cx + fx p_x/p_z,
//               y = cy - fy p_y/p_z; pixel (i, j) sampled at (i + 0.5, j + 0.5);
//               p_z <= near is not drawn;
//   projection  Sigma' = J R Sigma R^T J^T + 0.3 I (local affine approximation,
//               screen-space low-pass), Sigma = Rq diag(s^2) Rq^T;
//   alpha       min(0.99, sigma exp(-q/2)), q = delta^T Sigma'^-1 delta; a primitive
//               contributes to a pixel iff alpha >= 1/255;
//   order       by p_z, ties by primitive index;
//   stop        a pixel stops before the contribution that would take T below 1e-4.
//
// Pipeline (all on one stream): per-primitive projection and footprint (a square
// holding every pixel centre where alpha >= 1/255 can hold, so the image does not
// depend on the binning); a stable LSD radix sort (8-bit digits, written here) of
// the primitives by depth; an exclusive scan, in that order, of the tiles each
// primitive touches; emission of (tile, index) pairs in depth order; a stable
// radix sort of the pairs by tile alone (so each tile's list stays in depth order,
// ties by index); per-tile ranges; then one block per 16 x 16 tile: batches of 256
// primitives staged in shared memory, one thread per pixel. The backward walks
// each pixel's list back to front (T recovered by division), reduces the four
// per-primitive gradients over the warp in six shuffles and adds them with one
// atomic per warp, value and primitive. The forward reads the pair total once on
// the host to size the pair sort (one stream synchronisation).
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "nasg_host.h"
#include "nasg_vec.cuh"

namespace nasg {
namespace raster {

constexpr int kTile = 16;
constexpr int kTilePixels = kTile * kTile;
constexpr int kBlock = 256;
constexpr int kSortItems = 16;                    // keys per thread per sort block
constexpr int kSortChunk = kBlock * kSortItems;   // 4096 keys per sort block
constexpr int kScanChunk = 1024;                  // elements per scan block (4 per thread)
constexpr float kAlphaMin = 1.f / 255.f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kLowPass = 0.3f;
constexpr float kLog2e = 1.44269504088896341f;

struct Cam {
  float r[9], c[3], fx, fy, cx, cy, near_z;
  int w, h, tx, ty;
};

// Workspace layout (byte offsets, each 256-aligned), from n, tiles, pixels and the pair capacity.
struct Layout {
  size_t mean, conic, depth, rect, touched, offsets, scan_blocks, dkeys0, dkeys1, order0, order1, keys0, keys1, vals0,
      vals1, hist, ranges, ncontrib, header, total;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline Layout layout(int64_t n, int64_t tiles, int64_t pixels, int64_t cap) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
  const int64_t nscan = (n + kScanChunk - 1) / kScanChunk;
  const int64_t big = cap > n ? cap : n;
  const int64_t sblocks = (big + kSortChunk - 1) / kSortChunk;
  const int64_t hist = 256 * (sblocks > 0 ? sblocks : 1);
  L.header = take(256);
  L.mean = take(size_t(n) * sizeof(float2));
  L.conic = take(size_t(n) * sizeof(float4));
  L.depth = take(size_t(n) * sizeof(float));
  L.rect = take(size_t(n) * sizeof(int4));
  L.touched = take(size_t(n) * sizeof(uint32_t));
  L.offsets = take(size_t(n) * sizeof(uint32_t));
  L.scan_blocks = take(size_t(nscan + (hist + kScanChunk - 1) / kScanChunk + 2) * sizeof(uint32_t));
  L.dkeys0 = take(size_t(n) * sizeof(uint32_t));
  L.dkeys1 = take(size_t(n) * sizeof(uint32_t));
  L.order0 = take(size_t(n) * sizeof(uint32_t));
  L.order1 = take(size_t(n) * sizeof(uint32_t));
  L.keys0 = take(size_t(cap) * sizeof(uint32_t));
  L.keys1 = take(size_t(cap) * sizeof(uint32_t));
  L.vals0 = take(size_t(cap) * sizeof(uint32_t));
  L.vals1 = take(size_t(cap) * sizeof(uint32_t));
  L.hist = take(size_t(hist) * sizeof(uint32_t));
  L.ranges = take(size_t(tiles) * sizeof(uint2));
  L.ncontrib = take(size_t(pixels) * sizeof(uint32_t));
  L.total = o;
  return L;
}

// Header words in the workspace: the pair total (32-bit scan result and a 64-bit sum).
struct Header {
  uint32_t pairs;
  uint32_t pad;
  unsigned long long pairs64;
};

// Radix passes over the pairs' tile keys (8 bits each).
inline int sort_passes(int64_t tiles) {
  int tile_bits = 0;
  while ((int64_t(1) << tile_bits) < tiles) ++tile_bits;
  return tile_bits > 0 ? (tile_bits + 7) / 8 : 1;
}

// ---------------------------------------------------------------------------
// Projection and footprint
// ---------------------------------------------------------------------------

__global__ void project_kernel(int64_t n, const float* __restrict__ means, const float* __restrict__ scales,
                               const float* __restrict__ quats, const float* __restrict__ opacity, Cam cam,
                               float2* __restrict__ mean2, float4* __restrict__ conic, float* __restrict__ depth,
                               int4* __restrict__ rect, uint32_t* __restrict__ touched, uint32_t* __restrict__ dkey,
                               uint32_t* __restrict__ order) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t count = 0;
  int4 rc = make_int4(0, -1, 0, -1);
  const float mx = means[3 * i] - cam.c[0], my = means[3 * i + 1] - cam.c[1], mz = means[3 * i + 2] - cam.c[2];
  const float px = cam.r[0] * mx + cam.r[1] * my + cam.r[2] * mz;
  const float py = cam.r[3] * mx + cam.r[4] * my + cam.r[5] * mz;
  const float pz = cam.r[6] * mx + cam.r[7] * my + cam.r[8] * mz;
  const float sig = opacity[i];
  depth[i] = pz;
  if (pz > cam.near_z && sig * 255.f > 1.f) {
    const float iz = 1.f / pz;
    const float u = cam.cx + cam.fx * px * iz;
    const float v = cam.cy - cam.fy * py * iz;
    // J (2x3): rows (fx/z, 0, -fx x/z^2), (0, -fy/z, fy y/z^2); M = J R
    const float j00 = cam.fx * iz, j02 = -cam.fx * px * iz * iz;
    const float j11 = -cam.fy * iz, j12 = cam.fy * py * iz * iz;
    float m0[3], m1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      m0[c] = j00 * cam.r[c] + j02 * cam.r[6 + c];
      m1[c] = j11 * cam.r[3 + c] + j12 * cam.r[6 + c];
    }
    // Sigma = Rq diag(s^2) Rq^T from the normalised quaternion (w, x, y, z)
    float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
    const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= qn; qx *= qn; qy *= qn; qz *= qn;
    const float R[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                        2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                        2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
    const float s0 = scales[3 * i], s1 = scales[3 * i + 1], s2 = scales[3 * i + 2];
    const float ss[3] = {s0 * s0, s1 * s1, s2 * s2};
    // A = M Rq (2x3); Sigma' = A diag(s^2) A^T + 0.3 I
    float a0[3], a1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      a0[k] = m0[0] * R[k] + m0[1] * R[3 + k] + m0[2] * R[6 + k];
      a1[k] = m1[0] * R[k] + m1[1] * R[3 + k] + m1[2] * R[6 + k];
    }
    float sa = kLowPass, sb = 0.f, sc = kLowPass;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      sa += a0[k] * a0[k] * ss[k];
      sb += a0[k] * a1[k] * ss[k];
      sc += a1[k] * a1[k] * ss[k];
    }
    const float det = sa * sc - sb * sb;
    if (det > 0.f) {
      const float idet = 1.f / det;
      conic[i] = make_float4(sc * idet, -sb * idet, sa * idet, sig);
      mean2[i] = make_float2(u, v);
      // every pixel centre with alpha >= 1/255 lies within lambda_max * 2 ln(255 sigma)
      // of the mean; one pixel of slack for the FP32 evaluation
      const float half = 0.5f * (sa + sc);
      const float lmax = half + sqrtf(fmaxf(0.25f * (sa - sc) * (sa - sc) + sb * sb, 0.f));
      const float rad = sqrtf(lmax * 2.f * logf(255.f * sig)) + 1.f;
      // tile bounds clamped to [-1, tiles] before the integer conversion (u, v or rad may be huge)
      const float ftx = float(cam.tx), fty = float(cam.ty);
      const int x0 = max(0, int(fminf(fmaxf(floorf((u - rad - 0.5f) / kTile), -1.f), ftx)));
      const int x1 = min(cam.tx - 1, int(fminf(fmaxf(floorf((u + rad - 0.5f) / kTile), -1.f), ftx)));
      const int y0 = max(0, int(fminf(fmaxf(floorf((v - rad - 0.5f) / kTile), -1.f), fty)));
      const int y1 = min(cam.ty - 1, int(fminf(fmaxf(floorf((v + rad - 0.5f) / kTile), -1.f), fty)));
      if (x0 <= x1 && y0 <= y1 && isfinite(u) && isfinite(v) && isfinite(rad)) {
        rc = make_int4(x0, x1, y0, y1);
        count = uint32_t((x1 - x0 + 1) * (y1 - y0 + 1));
      }
    }
  }
  rect[i] = rc;
  touched[i] = count;
  // depth sort key: the bits of a positive float order like its value; primitives
  // that draw nothing go last
  dkey[i] = count ? __float_as_uint(pz) : 0xffffffffu;
  order[i] = uint32_t(i);
}

// ---------------------------------------------------------------------------
// Exclusive scan of uint32 (two levels: per-chunk sums, then one block over the sums)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_tot, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < int(blockDim.x >> 5) ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < int(blockDim.x >> 5)) warp_tot[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const uint32_t before = (warp > 0 ? warp_tot[warp - 1] : 0u) + inc - x;
  if (total) *total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

// out[i] = sum_{j < i} in[i] within each chunk of kScanChunk; sums[b] = chunk total.
__global__ void scan_chunks_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                                   uint32_t* __restrict__ sums) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t tot;
  const int64_t base = int64_t(blockIdx.x) * kScanChunk + int64_t(threadIdx.x) * 4;
  uint32_t v[4];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = base + k < n ? in[base + k] : 0u;
    s += v[k];
  }
  uint32_t run = block_exclusive_scan(s, warp_tot, &tot);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One block: exclusive scan of the chunk sums in place; total -> *total.
__global__ void scan_sums_kernel(uint32_t* __restrict__ sums, int64_t m, uint32_t* __restrict__ total) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t tot;
  uint32_t carry = 0;
  for (int64_t base = 0; base < m; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const uint32_t x = i < m ? sums[i] : 0u;
    const uint32_t ex = block_exclusive_scan(x, warp_tot, &tot);
    if (i < m) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// Sum of the per-primitive tile counts in 64 bits (the 32-bit scan wraps past 2^32).
__global__ void sum64_kernel(const uint32_t* __restrict__ in, int64_t n, unsigned long long* __restrict__ total) {
  unsigned long long v = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    v += in[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

__global__ void scan_add_kernel(uint32_t* __restrict__ out, int64_t n, const uint32_t* __restrict__ sums) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] += sums[i / kScanChunk];
}

// Exclusive scan of n uint32 values (in may equal out); total to *total (device).
static void exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* sums, uint32_t* total,
                           cudaStream_t s) {
  const int64_t chunks = (n + kScanChunk - 1) / kScanChunk;
  scan_chunks_kernel<<<unsigned(chunks), kBlock, 0, s>>>(in, out, n, sums);
  scan_sums_kernel<<<1, 1024, 0, s>>>(sums, chunks, total);
  scan_add_kernel<<<unsigned((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(out, n, sums);
}

// ---------------------------------------------------------------------------
// Pair emission, radix sort, tile ranges
// ---------------------------------------------------------------------------

// touched counts in depth order (for the scan that places each primitive's pairs)
__global__ void gather_counts_kernel(int64_t n, const uint32_t* __restrict__ order,
                                     const uint32_t* __restrict__ touched, uint32_t* __restrict__ out) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < n) out[k] = touched[order[k]];
}

// pairs (tile, primitive) of the k-th primitive in depth order, at offsets[k]
__global__ void emit_kernel(int64_t n, const uint32_t* __restrict__ order, const int4* __restrict__ rect,
                            const uint32_t* __restrict__ offsets, int tiles_x, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t i = order[k];
  const int4 r = rect[i];
  if (r.y < r.x) return;
  uint32_t o = offsets[k];
  for (int ty = r.z; ty <= r.w; ++ty)
    for (int tx = r.x; tx <= r.y; ++tx) {
      keys[o] = uint32_t(ty * tiles_x + tx);
      vals[o] = i;
      ++o;
    }
}

__global__ void radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t m, int shift,
                                  uint32_t* __restrict__ hist, int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kSortChunk;
#pragma unroll 4
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t j = base + int64_t(k) * kBlock + threadIdx.x;
    if (j < m) atomicAdd(&h[uint32_t(keys[j] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[int64_t(threadIdx.x) * nblocks + blockIdx.x] = h[threadIdx.x];  // digit-major
}

// Stable scatter of one block's chunk: rounds of 256 keys in order; within a
// round, keys with equal digits keep thread order (warp match + per-warp counts).
__global__ void radix_scatter_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                     uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t m, int shift,
                                     const uint32_t* __restrict__ offs, int nblocks) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t wcnt[kBlock / 32][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  run[threadIdx.x] = offs[int64_t(threadIdx.x) * nblocks + blockIdx.x];
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t base = int64_t(blockIdx.x) * kSortChunk;
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t j = base + int64_t(r) * kBlock + threadIdx.x;
    if (base + int64_t(r) * kBlock >= m) break;  // block-uniform
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const bool ok = j < m;
    uint32_t key = 0;
    uint32_t val = 0, d = 256;
    if (ok) {
      key = kin[j];
      val = vin[j];
      d = uint32_t(key >> shift) & 255u;
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    if (ok && lane == leader) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (ok) {
      uint32_t o = run[d] + __popc(peers & lt);
      for (int w = 0; w < warp; ++w) o += wcnt[w][d];
      kout[o] = key;
      vout[o] = val;
    }
    __syncthreads();
    uint32_t add = 0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) add += wcnt[w][threadIdx.x];
    run[threadIdx.x] += add;
    __syncthreads();
  }
}

__global__ void ranges_kernel(const uint32_t* __restrict__ keys, int64_t m, uint2* __restrict__ ranges) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const uint32_t t = keys[j];
  if (j == 0 || keys[j - 1] != t) ranges[t].x = uint32_t(j);
  if (j == m - 1 || keys[j + 1] != t) ranges[t].y = uint32_t(j + 1);
}

// Stable LSD radix sort of (key, value) pairs over the given 8-bit digits; returns
// the buffer index (0 or 1) that holds the result.
static int radix_sort(uint32_t* keys[2], uint32_t* vals[2], int64_t m, int passes, uint32_t* hist, uint32_t* sums,
                      cudaStream_t s) {
  int cur = 0;
  if (m <= 0) return cur;
  const int nblocks = int((m + kSortChunk - 1) / kSortChunk);
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = 8 * ps;
    radix_hist_kernel<<<nblocks, kBlock, 0, s>>>(keys[cur], m, shift, hist, nblocks);
    exclusive_scan(hist, hist, int64_t(256) * nblocks, sums, nullptr, s);
    radix_scatter_kernel<<<nblocks, kBlock, 0, s>>>(keys[cur], vals[cur], keys[1 - cur], vals[1 - cur], m, shift,
                                                    hist, nblocks);
    cur = 1 - cur;
  }
  return cur;
}

// ---------------------------------------------------------------------------
// Tile rendering
// ---------------------------------------------------------------------------

// alpha of a staged primitive at a pixel centre; 0 when below 1/255. Every
// operation is explicitly rounded so that the forward and the backward kernels
// take the same decisions on the same inputs.
__device__ __forceinline__ float pixel_alpha(float2 m, float4 k, float px, float py, float& rho) {
  const float dx = __fsub_rn(px, m.x), dy = __fsub_rn(py, m.y);
  const float q = __fmaf_rn(__fmul_rn(k.x, dx), dx,
                            __fmaf_rn(__fmul_rn(2.f * k.y, dx), dy, __fmul_rn(__fmul_rn(k.z, dy), dy)));
  rho = ex2a(__fmul_rn(__fmul_rn(-0.5f, q), kLog2e));
  const float a = fminf(kAlphaMax, __fmul_rn(k.w, rho));
  return a >= kAlphaMin ? a : 0.f;
}

__global__ void __launch_bounds__(kTilePixels) render_fwd_kernel(
    Cam cam, const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals, const float2* __restrict__ mean2,
    const float4* __restrict__ conic, const float* __restrict__ colours, float* __restrict__ image,
    float* __restrict__ final_t, uint32_t* __restrict__ ncontrib) {
  __shared__ float2 s_mean[kBlock];
  __shared__ float4 s_conic[kBlock];
  __shared__ float s_col[kBlock * 3];
  const int tile = blockIdx.x;
  const int tx = tile % cam.tx, ty = tile / cam.tx;
  const int pxi = tx * kTile + (threadIdx.x & (kTile - 1));
  const int pyi = ty * kTile + (threadIdx.x >> 4);
  const bool inside = pxi < cam.w && pyi < cam.h;
  const float px = float(pxi) + 0.5f, py = float(pyi) + 0.5f;
  const uint2 rg = ranges[tile];
  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  uint32_t last = 0;
  bool done = !inside;
  for (uint32_t b = rg.x; b < rg.y; b += kBlock) {
    if (__syncthreads_count(done) == kBlock) break;
    const uint32_t j = b + threadIdx.x;
    if (j < rg.y) {
      const uint32_t id = vals[j];
      s_mean[threadIdx.x] = mean2[id];
      s_conic[threadIdx.x] = conic[id];
      s_col[3 * threadIdx.x] = colours[3 * id];
      s_col[3 * threadIdx.x + 1] = colours[3 * id + 1];
      s_col[3 * threadIdx.x + 2] = colours[3 * id + 2];
    }
    __syncthreads();
    const int cnt = int(min(uint32_t(kBlock), rg.y - b));
    for (int k = 0; k < cnt && !done; ++k) {
      float rho;
      const float a = pixel_alpha(s_mean[k], s_conic[k], px, py, rho);
      if (a == 0.f) continue;
      const float test = T * (1.f - a);
      if (test < kTMin) {
        done = true;
        break;
      }
      const float w = a * T;
      c0 = fmaf(s_col[3 * k], w, c0);
      c1 = fmaf(s_col[3 * k + 1], w, c1);
      c2 = fmaf(s_col[3 * k + 2], w, c2);
      T = test;
      last = b - rg.x + uint32_t(k) + 1;
    }
  }
  if (inside) {
    const int64_t p = int64_t(pyi) * cam.w + pxi;
    image[3 * p] = c0;
    image[3 * p + 1] = c1;
    image[3 * p + 2] = c2;
    final_t[p] = T;
    ncontrib[p] = last;
  }
}

__global__ void __launch_bounds__(kTilePixels) render_bwd_kernel(
    Cam cam, const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals, const float2* __restrict__ mean2,
    const float4* __restrict__ conic, const float* __restrict__ colours, const float* __restrict__ final_t,
    const uint32_t* __restrict__ ncontrib, const float* __restrict__ g_image, float* __restrict__ g_colours,
    float* __restrict__ g_opacity) {
  __shared__ float2 s_mean[kBlock];
  __shared__ float4 s_conic[kBlock];
  __shared__ float s_col[kBlock * 3];
  __shared__ uint32_t s_id[kBlock];
  const int tile = blockIdx.x;
  const int tx = tile % cam.tx, ty = tile / cam.tx;
  const int pxi = tx * kTile + (threadIdx.x & (kTile - 1));
  const int pyi = ty * kTile + (threadIdx.x >> 4);
  const bool inside = pxi < cam.w && pyi < cam.h;
  const float px = float(pxi) + 0.5f, py = float(pyi) + 0.5f;
  const uint2 rg = ranges[tile];
  const int64_t p = int64_t(pyi) * cam.w + pxi;
  float T = inside ? final_t[p] : 1.f;
  const uint32_t last = inside ? ncontrib[p] : 0u;
  float g0 = 0.f, g1 = 0.f, g2 = 0.f;
  if (inside) {
    g0 = g_image[3 * p];
    g1 = g_image[3 * p + 1];
    g2 = g_image[3 * p + 2];
  }
  float af0 = 0.f, af1 = 0.f, af2 = 0.f;  // sum over later contributions of c alpha T
  const int lane = threadIdx.x & 31;
  // batches from the back of the range, starting at the block's furthest last
  // contribution (entries behind every pixel's stop point contribute nothing)
  __shared__ uint32_t s_last;
  if (threadIdx.x == 0) s_last = 0;
  __syncthreads();
  const uint32_t wl = __reduce_max_sync(0xffffffffu, last);
  if (lane == 0) atomicMax(&s_last, wl);
  __syncthreads();
  const uint32_t n = s_last;
  for (uint32_t done_cnt = 0; done_cnt < n; done_cnt += kBlock) {
    const uint32_t hi = n - done_cnt;                   // exclusive end (relative)
    const uint32_t lo = hi > uint32_t(kBlock) ? hi - kBlock : 0u;
    __syncthreads();
    const uint32_t jrel = lo + threadIdx.x;
    if (jrel < hi) {
      const uint32_t id = vals[rg.x + jrel];
      s_id[threadIdx.x] = id;
      s_mean[threadIdx.x] = mean2[id];
      s_conic[threadIdx.x] = conic[id];
      s_col[3 * threadIdx.x] = colours[3 * id];
      s_col[3 * threadIdx.x + 1] = colours[3 * id + 1];
      s_col[3 * threadIdx.x + 2] = colours[3 * id + 2];
    }
    __syncthreads();
    for (int k = int(hi - lo) - 1; k >= 0; --k) {
      const uint32_t pos = lo + uint32_t(k);  // position in the tile's list
      float rho = 0.f, a = 0.f;
      if (pos < last) a = pixel_alpha(s_mean[k], s_conic[k], px, py, rho);
      float gc0 = 0.f, gc1 = 0.f, gc2 = 0.f, go = 0.f;
      if (a > 0.f) {
        const float inv = 1.f / (1.f - a);
        const float Tb = T * inv;  // transmittance in front of this contribution
        const float w = a * Tb;
        gc0 = w * g0;
        gc1 = w * g1;
        gc2 = w * g2;
        const float c0 = s_col[3 * k], c1 = s_col[3 * k + 1], c2 = s_col[3 * k + 2];
        const float da = g0 * (c0 * Tb - af0 * inv) + g1 * (c1 * Tb - af1 * inv) + g2 * (c2 * Tb - af2 * inv);
        if (s_conic[k].w * rho < kAlphaMax) go = da * rho;
        af0 = fmaf(c0, w, af0);
        af1 = fmaf(c1, w, af1);
        af2 = fmaf(c2, w, af2);
        T = Tb;
      }
      if (__any_sync(0xffffffffu, a > 0.f)) {
        // four sums over the warp in six shuffles: halves exchange two values, then
        // quarters one, then a plain butterfly; lane 8 q (q = 0..3) ends with sum q
        const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
        float k0 = hi16 ? gc2 : gc0, k1 = hi16 ? go : gc1;
        const float s0 = hi16 ? gc0 : gc2, s1 = hi16 ? gc1 : go;
        k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
        k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
        float v = hi8 ? k1 : k0;
        v += __shfl_xor_sync(0xffffffffu, hi8 ? k0 : k1, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        if ((lane & 7) == 0) {
          const uint32_t id = s_id[k];
          const int q = lane >> 3;  // 0, 1, 2: colour channel; 3: opacity
          atomicAdd(q < 3 ? g_colours + 3 * id + q : g_opacity + id, v);
        }
      }
    }
  }
}

inline Cam make_cam(const nasg_raster_camera* c) {
  Cam k;
  for (int j = 0; j < 9; ++j) k.r[j] = c->rot[j];
  for (int j = 0; j < 3; ++j) k.c[j] = c->centre[j];
  k.fx = c->fx;
  k.fy = c->fy;
  k.cx = c->cx;
  k.cy = c->cy;
  k.near_z = c->near_z;
  k.w = c->width;
  k.h = c->height;
  k.tx = (c->width + kTile - 1) / kTile;
  k.ty = (c->height + kTile - 1) / kTile;
  return k;
}

inline bool camera_ok(const nasg_raster_camera* c) {
  if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384) return false;
  if (!(c->fx > 0.f) || !(c->fy > 0.f) || !(c->near_z > 0.f)) return false;
  for (int j = 0; j < 9; ++j)
    if (!std::isfinite(c->rot[j])) return false;
  return std::isfinite(c->cx) && std::isfinite(c->cy) && std::isfinite(c->centre[0]) &&
         std::isfinite(c->centre[1]) && std::isfinite(c->centre[2]);
}

}  // namespace raster
}  // namespace nasg

using namespace nasg;
using namespace nasg::raster;

extern "C" size_t nasg_raster_workspace_bytes(int64_t n, int32_t width, int32_t height, int64_t max_pairs) {
  if (n < 0 || n >= (int64_t(1) << 31) || width < 1 || height < 1 || width > 16384 || height > 16384 ||
      max_pairs < 0 || max_pairs >= (int64_t(1) << 32))
    return 0;
  const int64_t tiles = int64_t((width + kTile - 1) / kTile) * ((height + kTile - 1) / kTile);
  return layout(n, tiles, int64_t(width) * height, max_pairs).total;
}

extern "C" nasg_status nasg_raster_forward(int64_t n, const float* means, const float* scales, const float* quats,
                                           const float* opacity, const float* colours,
                                           const nasg_raster_camera* camera, float* image, float* final_t,
                                           int64_t max_pairs, void* workspace, size_t workspace_bytes,
                                           int64_t* n_pairs, void* stream) {
  if (!camera) return NASG_ERR_NULL;
  if (!camera_ok(camera)) return NASG_ERR_RANGE;
  if (n < 0 || n >= (int64_t(1) << 31) || max_pairs < 0 || max_pairs >= (int64_t(1) << 32)) return NASG_ERR_RANGE;
  if (!image || !final_t || !workspace) return NASG_ERR_NULL;
  if (n > 0 && (!means || !scales || !quats || !opacity || !colours)) return NASG_ERR_NULL;
  if (!aligned(workspace, 256) || !aligned(means, 4) || !aligned(image, 4) || !aligned(final_t, 4))
    return NASG_ERR_ALIGN;
  const Cam cam = make_cam(camera);
  const int64_t tiles = int64_t(cam.tx) * cam.ty;
  const int64_t pixels = int64_t(cam.w) * cam.h;
  const Layout L = layout(n, tiles, pixels, max_pairs);
  if (workspace_bytes < L.total) return NASG_ERR_RANGE;
  cudaStream_t s = as_stream(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  Header* hdr = reinterpret_cast<Header*>(ws + L.header);
  auto* mean2 = reinterpret_cast<float2*>(ws + L.mean);
  auto* con = reinterpret_cast<float4*>(ws + L.conic);
  auto* dep = reinterpret_cast<float*>(ws + L.depth);
  auto* rect = reinterpret_cast<int4*>(ws + L.rect);
  auto* touched = reinterpret_cast<uint32_t*>(ws + L.touched);
  auto* offsets = reinterpret_cast<uint32_t*>(ws + L.offsets);
  auto* sums = reinterpret_cast<uint32_t*>(ws + L.scan_blocks);
  uint32_t* keys[2] = {reinterpret_cast<uint32_t*>(ws + L.keys0), reinterpret_cast<uint32_t*>(ws + L.keys1)};
  uint32_t* dkeys[2] = {reinterpret_cast<uint32_t*>(ws + L.dkeys0), reinterpret_cast<uint32_t*>(ws + L.dkeys1)};
  uint32_t* order[2] = {reinterpret_cast<uint32_t*>(ws + L.order0), reinterpret_cast<uint32_t*>(ws + L.order1)};
  uint32_t* vals[2] = {reinterpret_cast<uint32_t*>(ws + L.vals0), reinterpret_cast<uint32_t*>(ws + L.vals1)};
  auto* hist = reinterpret_cast<uint32_t*>(ws + L.hist);
  auto* ranges = reinterpret_cast<uint2*>(ws + L.ranges);
  auto* ncontrib = reinterpret_cast<uint32_t*>(ws + L.ncontrib);

  if (cudaMemsetAsync(hdr, 0, sizeof(Header), s) != cudaSuccess) return check_launch();
  if (cudaMemsetAsync(ranges, 0, size_t(tiles) * sizeof(uint2), s) != cudaSuccess) return check_launch();
  unsigned long long total64 = 0;
  int dcur = 0;
  if (n > 0) {
    project_kernel<<<unsigned((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, means, scales, quats, opacity, cam,
                                                                            mean2, con, dep, rect, touched, dkeys[0],
                                                                            order[0]);
    // primitives by depth (ties by index: the sort is stable), then their tile counts in that order
    dcur = radix_sort(dkeys, order, n, 4, hist, sums, s);
    gather_counts_kernel<<<unsigned((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, order[dcur], touched, offsets);
    exclusive_scan(offsets, offsets, n, sums, &hdr->pairs, s);
    sum64_kernel<<<unsigned(std::min<int64_t>((n + kBlock - 1) / kBlock, 1024)), kBlock, 0, s>>>(touched, n,
                                                                                                 &hdr->pairs64);
    if (cudaMemcpyAsync(&total64, &hdr->pairs64, sizeof(total64), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return check_launch();
  }
  if (n_pairs) *n_pairs = int64_t(total64);
  if (int64_t(total64) > max_pairs) return NASG_ERR_CAPACITY;
  const uint32_t total = uint32_t(total64);
  const int passes = sort_passes(tiles);
  int cur = 0;
  if (total > 0) {
    emit_kernel<<<unsigned((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, order[dcur], rect, offsets, cam.tx,
                                                                         keys[0], vals[0]);
    cur = radix_sort(keys, vals, total, passes, hist, sums, s);
    if (cur != passes % 2) return NASG_ERR_DEVICE;  // the backward relies on this parity
    ranges_kernel<<<unsigned((total + kBlock - 1) / kBlock), kBlock, 0, s>>>(keys[cur], total, ranges);
  }
  render_fwd_kernel<<<unsigned(tiles), kTilePixels, 0, s>>>(cam, ranges, vals[cur], mean2, con, colours, image,
                                                            final_t, ncontrib);
  return check_launch();
}

extern "C" nasg_status nasg_raster_backward(int64_t n, const float* colours, const nasg_raster_camera* camera,
                                            const float* final_t, const float* g_image, float* g_colours,
                                            float* g_opacity, int64_t max_pairs, void* workspace,
                                            size_t workspace_bytes, void* stream) {
  if (!camera) return NASG_ERR_NULL;
  if (!camera_ok(camera)) return NASG_ERR_RANGE;
  if (n < 0 || n >= (int64_t(1) << 31) || max_pairs < 0 || max_pairs >= (int64_t(1) << 32)) return NASG_ERR_RANGE;
  if (!final_t || !g_image || !workspace || !g_colours || !g_opacity) return NASG_ERR_NULL;
  if (n > 0 && !colours) return NASG_ERR_NULL;
  if (!aligned(workspace, 256)) return NASG_ERR_ALIGN;
  const Cam cam = make_cam(camera);
  const int64_t tiles = int64_t(cam.tx) * cam.ty;
  const Layout L = layout(n, tiles, int64_t(cam.w) * cam.h, max_pairs);
  if (workspace_bytes < L.total) return NASG_ERR_RANGE;
  cudaStream_t s = as_stream(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  if (cudaMemsetAsync(g_colours, 0, size_t(n) * 3 * sizeof(float), s) != cudaSuccess ||
      cudaMemsetAsync(g_opacity, 0, size_t(n) * sizeof(float), s) != cudaSuccess)
    return check_launch();
  if (n == 0) return NASG_OK;
  // the forward's sort ends in buffer (passes % 2)
  const uint32_t* vals = reinterpret_cast<const uint32_t*>(ws + (sort_passes(tiles) % 2 ? L.vals1 : L.vals0));
  render_bwd_kernel<<<unsigned(tiles), kTilePixels, 0, s>>>(
      cam, reinterpret_cast<const uint2*>(ws + L.ranges), vals, reinterpret_cast<const float2*>(ws + L.mean),
      reinterpret_cast<const float4*>(ws + L.conic), colours, final_t,
      reinterpret_cast<const uint32_t*>(ws + L.ncontrib), g_image, g_colours, g_opacity);
  return check_launch();
}
