// Plans for moving one contiguous span of a global buffer into shared memory
// with bulk asynchronous copies, whose source, destination and size must be
// multiples of 16 bytes, when the span's own start and length are not.
//
// The copy starts at the 16-byte boundary at or below the span's first byte
// and ends at the boundary at or above its last byte, unless that would read
// past the end of the buffer: then the bulk copy stops at the boundary below
// the span's end and the remaining bytes (fewer than 16) are moved by plain
// loads. The span then sits `head` bytes into the destination. Offsets are in
// bytes from the buffer's base, which must itself be 16-byte aligned.
//
// Also the shared-memory stage layout of the staged evaluation kernel and the
// plans of one of its tiles. Pure integer arithmetic, shared by the kernels and
// a host-side check of every plan's alignment and bounds.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define NASG_HD __host__ __device__ __forceinline__
#else
#define NASG_HD inline
#endif

namespace nasg {

struct SpanPlan {
  uint64_t src;   // offset of the first copied byte (multiple of 16)
  uint32_t bulk;  // bytes moved by the bulk copy (multiple of 16; 0 for none)
  uint32_t tail;  // bytes moved by plain loads, from offset src + bulk (< 16, even)
  uint32_t head;  // the span's first byte sits at destination + head (< 16)
};

// Span [off, off + bytes) of a buffer of buf_bytes bytes; off, bytes and
// buf_bytes even, off + bytes <= buf_bytes.
NASG_HD SpanPlan span_plan(uint64_t off, uint32_t bytes, uint64_t buf_bytes) {
  SpanPlan s;
  s.src = off & ~uint64_t(15);
  s.head = uint32_t(off - s.src);
  const uint64_t end = off + bytes;
  const uint64_t up = (end + 15) & ~uint64_t(15);
  if (up <= buf_bytes) {
    s.bulk = uint32_t(up - s.src);
    s.tail = 0;
  } else {
    const uint64_t dn = end & ~uint64_t(15);
    s.bulk = dn > s.src ? uint32_t(dn - s.src) : 0u;
    s.tail = uint32_t(end - s.src) - s.bulk;
  }
  return s;
}

// Destination bytes that hold any plan of a span of at most `bytes` bytes
// (a head below 16 plus rounding below 16), a multiple of 16.
NASG_HD constexpr uint32_t span_capacity(uint32_t bytes) { return (bytes + 30u + 15u) & ~15u; }

// ---------------------------------------------------------------------------
// Tiles of the staged evaluation kernel
// ---------------------------------------------------------------------------

struct TileGeom {
  uint32_t tp;          // primitives per tile
  uint32_t plane_bytes; // bytes of one parameter plane's span in a stage
  uint32_t mu_cap;      // bytes of the means / upstream-gradient regions
  uint32_t c0_cap;      // bytes of one diffuse-colour plane's region
  uint32_t off_mu, off_gc, off_c0, stage_bytes;
};

// Parameter spans are whole 16-byte units (N L sizeof(T) % 16 == 0, checked on
// the host; tp L sizeof(T) is a multiple of 32 for even L). ANYN false: N % 8
// == 0, so every span of every tile is whole 16-byte units at 16-byte
// boundaries and the regions are packed. ANYN true (any N): the means, upstream
// gradients and diffuse colours follow span plans, so their regions hold a
// plan's head and rounding.
template <typename T, int P, bool ANYN>
NASG_HD constexpr TileGeom tile_geom(int slice_log2, int n_lobes, uint32_t threads = 256u) {
  TileGeom g{};
  g.tp = threads >> slice_log2;
  g.plane_bytes = g.tp * uint32_t(n_lobes) * uint32_t(sizeof(T));
  g.mu_cap = ANYN ? span_capacity(g.tp * 12u) : g.tp * 12u;
  g.c0_cap = ANYN ? span_capacity(g.tp * uint32_t(sizeof(T))) : g.tp * uint32_t(sizeof(T));
  g.off_mu = P * g.plane_bytes;
  g.off_gc = g.off_mu + g.mu_cap;
  g.off_c0 = g.off_gc + g.mu_cap;
  g.stage_bytes = (g.off_c0 + 3u * g.c0_cap + 127u) & ~127u;
  return g;
}

// Byte offset, within its stage region, of diffuse-colour plane c of any tile:
// a tile's first primitive p0 is a multiple of tp >= 8, so (c N + p0) sizeof(T)
// = c N sizeof(T) modulo 16. (The means and upstream gradients start at 12 p0,
// a multiple of 16: no offset.)
template <typename T, bool ANYN = true>
NASG_HD uint32_t c0_head(uint32_t c, uint64_t n) {
  return ANYN ? (c * uint32_t(n & 15u) * uint32_t(sizeof(T))) & 15u : 0u;
}

// Plans of the means / upstream-gradient spans (one plan for both: records of
// 12 bytes, buffers of 12 N bytes) and of the three diffuse-colour spans
// (planes [3][N] of sizeof(T)) of `count` primitives from p0.
struct PrimPlans {
  SpanPlan mu;
  SpanPlan c0[3];
};

template <typename T>
NASG_HD PrimPlans prim_plans(uint64_t n, uint64_t p0, uint32_t count) {
  PrimPlans r;
  r.mu = span_plan(p0 * 12u, count * 12u, n * 12u);
  for (uint32_t c = 0; c < 3; ++c)
    r.c0[c] = span_plan((c * n + p0) * sizeof(T), count * uint32_t(sizeof(T)), 3u * n * sizeof(T));
  return r;
}

// The same plans for a unit of `count` primitives from p0 whose first primitive
// is a multiple of 8: when the unit is followed by at least 16 more primitives,
// the means span is exact (12 p0 is a multiple of 16) and a diffuse-colour span
// rounded out to 16-byte boundaries ends inside its buffer, which needs no
// comparisons; otherwise the general plans.
template <typename T>
NASG_HD PrimPlans unit_plans(uint64_t n, uint64_t p0, uint32_t count) {
  if (p0 + count + 16u > n) return prim_plans<T>(n, p0, count);
  constexpr uint32_t es = uint32_t(sizeof(T));
  PrimPlans r;
  r.mu = SpanPlan{p0 * 12u, count * 12u, 0u, 0u};
  for (uint32_t c = 0; c < 3; ++c) {
    const uint32_t head = c0_head<T>(c, n);
    r.c0[c] = SpanPlan{(c * n + p0) * es - head, count * es + (head ? 16u : 0u), 0u, head};
  }
  return r;
}

// The copies of one tile, numbered j = 0 .. P + 4: j < P parameter plane j
// (element j N L + p0 L on), j = P the means, j = P + 1 the upstream gradients
// (the means' plan), j = P + 2 + c diffuse-colour plane c. tile_span gives copy
// j's plan (byte offsets from its buffer's base), tile_dst its region in the
// stage. Offsets below 2^32 are formed in 32 bits: the staged kernel takes
// P N L < 2^31 elements.
template <typename T, int P>
NASG_HD uint32_t tile_dst(const TileGeom& g, uint32_t j) {
  return j < uint32_t(P) ? j * g.plane_bytes
         : j == uint32_t(P) ? g.off_mu
         : j == uint32_t(P) + 1u ? g.off_gc
                                 : g.off_c0 + (j - uint32_t(P) - 2u) * g.c0_cap;
}

template <typename T, int P, bool ANYN>
NASG_HD SpanPlan tile_span(const TileGeom& g, uint32_t n, uint32_t n_lobes, uint32_t tile, uint32_t j) {
  constexpr uint32_t es = uint32_t(sizeof(T));
  const uint32_t p0 = tile * g.tp;
  const uint32_t count = n - p0 < g.tp ? n - p0 : g.tp;
  if (j < uint32_t(P))  // whole 16-byte units (N L sizeof(T) % 16 == 0)
    return SpanPlan{(uint64_t(j) * n + p0) * n_lobes * es, count * n_lobes * es, 0u, 0u};
  // an inner tile (full, with at least 16 primitives after it): the means span is
  // exact, and a diffuse-colour span rounded out to 16-byte boundaries ends
  // inside its buffer
  const bool inner = p0 + g.tp + 16u <= n;
  if (j <= uint32_t(P) + 1u) {
    if (!ANYN || inner) return SpanPlan{uint64_t(p0) * 12u, count * 12u, 0u, 0u};
    return span_plan(uint64_t(p0) * 12u, count * 12u, uint64_t(n) * 12u);
  }
  const uint32_t c = j - uint32_t(P) - 2u;
  if (!ANYN) return SpanPlan{uint64_t((c * n + p0) * es), count * es, 0u, 0u};  // N % 8 == 0: exact
  if (inner) {
    const uint32_t head = c0_head<T>(c, n);
    return SpanPlan{uint64_t((c * n + p0) * es - head), g.tp * es + (head ? 16u : 0u), 0u, head};
  }
  return span_plan((uint64_t(c) * n + p0) * es, count * es, uint64_t(3) * n * es);
}

// Items per thread in a sub-tile of the batched kernels: two for BF16 parameters
// (sub-tiles of 2 x 256/S primitives), one for FP32 (whose stages are twice as large).
template <typename T>
NASG_HD constexpr int unit_items() { return sizeof(T) == 2 ? 2 : 1; }
NASG_HD constexpr int unit_items_of(int param_dtype) { return param_dtype == 1 ? 2 : 1; }  // NASG_DTYPE_BF16

// Stage layout of the staged batched kernel: room for the sub-tile of any scene it
// stages (L >= 4, so S >= 2: at most I x 128 primitives and I x 512 lobes), i.e. the
// layout of an I x 128-primitive tile of four lobes.
template <typename T, int P>
NASG_HD constexpr TileGeom batch_geom() { return tile_geom<T, P, true>(1, 4, 256u * uint32_t(unit_items<T>())); }

}  // namespace nasg
