// Host-side check of the staged kernels' copy plans (csrc/nasg_span.h): for
// every tile of every eligible (N, L, element size) in a sweep, each bulk copy
// starts on a 16-byte boundary at a 16-byte aligned destination, moves a
// multiple of 16 bytes and stays inside its buffer; the plain-load tail is
// shorter than 16 bytes and inside the buffer; bulk + tail cover the span; the
// destination region holds them; and the offsets the consumers assume (heads
// of the means and diffuse-colour regions) are the plans' heads.
// Prints "ok <cases>" and exits 0, or prints the first failure and exits 1.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "nasg_span.h"

using namespace nasg;

static long g_cases = 0;

#define CHECK(cond, ...)                                            \
  do {                                                              \
    if (!(cond)) {                                                  \
      std::printf("FAIL %s: ", #cond);                              \
      std::printf(__VA_ARGS__);                                     \
      std::printf("\n");                                            \
      std::exit(1);                                                 \
    }                                                               \
  } while (0)

static void check_span(const SpanPlan& s, uint64_t off, uint32_t bytes, uint64_t buf, uint32_t cap,
                       uint32_t dst_off, const char* what, uint32_t n, uint32_t L, uint32_t tile) {
  CHECK(s.src % 16 == 0, "%s n=%u L=%u tile=%u", what, n, L, tile);
  CHECK(s.bulk % 16 == 0, "%s n=%u L=%u tile=%u", what, n, L, tile);
  CHECK(dst_off % 16 == 0, "%s n=%u L=%u tile=%u", what, n, L, tile);
  CHECK(s.src + s.bulk <= buf, "%s n=%u L=%u tile=%u", what, n, L, tile);
  CHECK(s.tail < 16 && s.tail % 2 == 0, "%s n=%u L=%u tile=%u tail=%u", what, n, L, tile, s.tail);
  CHECK(s.src + s.bulk + s.tail <= buf, "%s n=%u L=%u tile=%u", what, n, L, tile);
  CHECK(s.src + s.head == off, "%s n=%u L=%u tile=%u", what, n, L, tile);
  CHECK(s.head + bytes <= s.bulk + s.tail, "%s n=%u L=%u tile=%u", what, n, L, tile);
  CHECK(s.bulk + s.tail <= cap, "%s n=%u L=%u tile=%u", what, n, L, tile);
  ++g_cases;
}

// Tiles of the staged kernels for a block of `threads` x items per thread (256: the passes with
// a backward, 384: the forward alone, 512 / 768: two / three items per thread of 256-thread blocks).
template <typename T, int P, bool ANYN>
static void check_eval(uint32_t n, uint32_t L, uint32_t threads = 256u) {
  const uint32_t es = sizeof(T);
  int slog = 0;
  while ((1u << slog) < (L + 1) / 2) ++slog;
  const TileGeom g = tile_geom<T, P, ANYN>(slog, int(L), threads);
  CHECK(g.off_mu % 16 == 0 && g.off_gc % 16 == 0 && g.off_c0 % 16 == 0 && g.c0_cap % 16 == 0 &&
            g.stage_bytes % 128 == 0 && g.off_c0 + 3 * g.c0_cap <= g.stage_bytes,
        "layout L=%u", L);
  const uint64_t NL = uint64_t(n) * L;
  const uint32_t n_tiles = (n + g.tp - 1) / g.tp;
  for (uint32_t tile = 0; tile < n_tiles; ++tile) {
    const uint32_t p0 = tile * g.tp;
    const uint32_t count = n - p0 < g.tp ? n - p0 : g.tp;
    CHECK(count >= 1 && count <= g.tp, "count n=%u L=%u tile=%u", n, L, tile);
    for (uint32_t j = 0; j < uint32_t(P) + 5u; ++j) {
      const SpanPlan sp = tile_span<T, P, ANYN>(g, n, L, tile, j);
      const uint32_t dst = tile_dst<T, P>(g, j);
      if (j < uint32_t(P)) {
        const uint64_t off = (uint64_t(j) * NL + uint64_t(p0) * L) * es;
        CHECK(sp.src == off && sp.head == 0 && sp.tail == 0 && sp.bulk == count * L * es, "param n=%u L=%u tile=%u",
              n, L, tile);
        CHECK(off % 16 == 0 && sp.bulk % 16 == 0 && off + sp.bulk <= uint64_t(P) * NL * es && sp.bulk <= g.plane_bytes &&
                  dst % 16 == 0 && dst + g.plane_bytes <= g.off_mu,
              "param n=%u L=%u tile=%u", n, L, tile);
      } else if (j <= uint32_t(P) + 1u) {
        check_span(sp, uint64_t(p0) * 12, count * 12, uint64_t(n) * 12, g.mu_cap, dst, "mu", n, L, tile);
        CHECK(sp.head == 0, "mu head n=%u L=%u tile=%u", n, L, tile);
        CHECK(dst == (j == uint32_t(P) ? g.off_mu : g.off_gc), "mu dst");
      } else {
        const uint32_t c = j - uint32_t(P) - 2u;
        check_span(sp, (uint64_t(c) * n + p0) * es, count * es, uint64_t(3) * n * es, g.c0_cap, dst, "c0", n, L, tile);
        CHECK(sp.head == (c0_head<T, ANYN>(c, n)), "c0 head n=%u L=%u tile=%u c=%u", n, L, tile, c);
        CHECK(dst == g.off_c0 + c * g.c0_cap, "c0 dst");
      }
    }
  }
}

// Units of the staged batched kernel: sub-tiles of I x 256/S primitives of one scene,
// staged into the fixed batch layout.
template <typename T, int P>
static void check_batch(uint32_t n, uint32_t L) {
  const uint32_t es = sizeof(T);
  int slog = 0;
  while ((1u << slog) < (L + 1) / 2) ++slog;
  const uint32_t tp = (256u >> slog) * uint32_t(unit_items<T>());
  const TileGeom g = batch_geom<T, P>();
  CHECK(g.off_mu % 16 == 0 && g.off_gc % 16 == 0 && g.off_c0 % 16 == 0 && g.c0_cap % 16 == 0 &&
            g.stage_bytes % 128 == 0 && g.off_c0 + 3 * g.c0_cap <= g.stage_bytes,
        "batch layout");
  const uint64_t NL = uint64_t(n) * L;
  for (uint64_t p0 = 0; p0 < n; p0 += tp) {
    const uint32_t count = uint32_t(n - p0 < tp ? n - p0 : tp);
    const uint32_t bytes = count * L * es;
    CHECK(bytes <= g.plane_bytes && bytes % 16 == 0, "batch params n=%u L=%u p0=%llu", n, L, (unsigned long long)p0);
    for (int p = 0; p < P; ++p)
      CHECK(((uint64_t(p) * NL + p0 * L) * es) % 16 == 0, "batch param start n=%u L=%u", n, L);
    const PrimPlans pp = unit_plans<T>(n, p0, count);
    const uint32_t tile = uint32_t(p0 / tp);
    check_span(pp.mu, p0 * 12, count * 12, uint64_t(n) * 12, g.mu_cap, g.off_mu, "batch mu", n, L, tile);
    CHECK(pp.mu.head == 0, "batch mu head n=%u L=%u", n, L);
    for (uint32_t c = 0; c < 3; ++c) {
      check_span(pp.c0[c], (uint64_t(c) * n + p0) * es, count * es, uint64_t(3) * n * es, g.c0_cap,
                 g.off_c0 + c * g.c0_cap, "batch c0", n, L, tile);
      CHECK(pp.c0[c].head == c0_head<T>(c, n), "batch c0 head n=%u L=%u c=%u", n, L, c);
    }
  }
}

struct F16 { uint16_t v; };

int main() {
  std::vector<uint32_t> ns;
  for (uint32_t n = 1; n <= 1200; ++n) ns.push_back(n);
  for (uint32_t k = 11; k <= 20; ++k)
    for (int d = -9; d <= 9; ++d) ns.push_back((1u << k) + d);
  const uint32_t big[] = {999983, 1000000, 1000003, 1833537, 2398541, 5000001};
  for (uint32_t n : big) ns.push_back(n);
  for (uint32_t L = 2; L <= 32; L += 2) {
    for (uint32_t n : ns) {
      if (uint64_t(n) * L * 11 >= (uint64_t(1) << 31)) continue;
      // the kernels take the packed layout (ANYN false) exactly when N % 8 == 0
      if ((uint64_t(n) * L * 2) % 16 == 0) {
        check_eval<F16, 10, true>(n, L);
        check_eval<F16, 9, true>(n, L);
        check_eval<F16, 11, true>(n, L);
        if (n % 8 == 0) check_eval<F16, 10, false>(n, L);
        const uint32_t many = L >= 8 ? 768u : 512u;
        check_eval<F16, 10, true>(n, L, many);
        check_eval<F16, 9, true>(n, L, many);
        if (n % 8 == 0) check_eval<F16, 10, false>(n, L, many);
      }
      if ((uint64_t(n) * L * 4) % 16 == 0) {
        check_eval<float, 10, true>(n, L);
        check_eval<float, 8, true>(n, L);
        if (n % 8 == 0) check_eval<float, 10, false>(n, L);
        check_eval<float, 10, true>(n, L, 384u);
        if (n % 8 == 0) check_eval<float, 10, false>(n, L, 384u);
        check_eval<float, 10, true>(n, L, 512u);
        if (n % 8 == 0) check_eval<float, 10, false>(n, L, 512u);
      }
      // batched scenes are staged when L >= 4 is even and N L sizeof(T) % 16 == 0
      if (L >= 4 && (uint64_t(n) * L * 2) % 16 == 0) check_batch<F16, 10>(n, L);
      if (L >= 4 && (uint64_t(n) * L * 4) % 16 == 0) check_batch<float, 9>(n, L);
    }
  }
  std::printf("ok %ld\n", g_cases);
  return 0;
}
