// FP32 elementary functions for the NASGabor kernels, generic over the value
// type V (float, or the packed pair P2 of nasg_vec.cuh), written from their
// series definitions and the hardware ex2/lg2/rcp approximations (no vendor
// math code). Each is checked on the GPU against float64 references through
// the library's math probe (tests/test_gpu_math.py).
//
//   vexp(x)       2^(x log2 e) by ex2.approx (relative error ~2^-22 plus the
//                 rounding of x log2 e, i.e. ~|x| 6e-8).
//   vexpm1n(y)    e^y - 1 for y <= 0: Taylor polynomial to y^8 on [-0.5, 0]
//                 (truncation < 1.1e-8 relative), 2^(y log2 e) - 1 below -0.5
//                 (|result| >= 0.39 there, so the subtraction loses nothing).
//   vtanh(x)      odd Taylor series to x^9 for |x| < 1/4, else
//                 (1 - e)/(1 + e) with e = e^{-2|x|}; 1 - tanh^2 x = 4 e/(1 + e)^2;
//                 tanh_lookup the same values by table for BF16-valued arguments.
//   vlnkappa(t)   ln(1 + t) for t in [-1, 0]: 2 atanh(t/(2 + t)) series to
//                 s^7 where 1 + t >= 0.75 (|s| <= 1/7: truncation < 1.9e-8 relative),
//                 lg2.approx elsewhere.
//   vcarrier(x)   cos^2 x and sin 2x (the NASGabor carrier and its slope) for
//                 |x| <= 6400; vsincos(x) gives sin x, cos x from the same
//                 Cody-Waite reduction x = n pi/2 + r with pi/2 split in three
//                 float parts (the first two with 12 significant bits, so n*C1
//                 and n*C2 are exact) and the Taylor polynomials of sin (to r^9)
//                 and cos (to r^10) on |r| <= pi/4 (truncation < 3e-9).
//   vcarrier_sum(y, w)  cos^2(y + w) and sin 2(y + w) by angle addition (the
//                 phase-shifted carrier, y = phi/2, w = k v/2).
#pragma once

#include "nasg_vec.cuh"

namespace nasg {

constexpr float kLog2e = 1.44269504088896341f;
constexpr float kLn2 = 0.693147180559945309f;

// 1/n! rounded to float
constexpr float kF2 = 0.5f, kF3 = 1.f / 6.f, kF4 = 1.f / 24.f, kF5 = 1.f / 120.f, kF6 = 1.f / 720.f,
                kF7 = 1.f / 5040.f, kF8 = 1.f / 40320.f, kF9 = 1.f / 362880.f;

template <class V>
__device__ __forceinline__ V vexp(V x) {
  return vex2(x * kLog2e);
}


template <class V>
__device__ __forceinline__ V taylor_expm1(V y) {
  V p = vfma(y, kF8, kF7);
  p = vfma(p, y, kF6);
  p = vfma(p, y, kF5);
  p = vfma(p, y, kF4);
  p = vfma(p, y, kF3);
  p = vfma(p, y, kF2);
  p = vfma(p, y, 1.f);
  return p * y;
}

template <class V>
__device__ __forceinline__ V vexpm1n(V y) {
  return vsel(vgt(y, -0.5f), taylor_expm1(y), vex2(y * kLog2e) - 1.f);
}

// e^y and e^y - 1 for y <= 0, each to full relative accuracy: below -1/2 both from
// 2^(y log2 e) (e^y - 1 <= -0.39 there), above from the Taylor polynomial (e^y >= 0.6).
// (e^y recovered as (e^y - 1) + 1 would keep no digits where e^y is tiny.)
template <class V>
__device__ __forceinline__ void vexp_expm1n(V y, V& e, V& em1) {
  const V ex = vex2(y * kLog2e);
  const V tl = taylor_expm1(y);
  const auto small = vgt(y, -0.5f);
  em1 = vsel(small, tl, ex - 1.f);
  e = vsel(small, tl + 1.f, ex);
}

template <class V>
__device__ __forceinline__ void vtanh(V x, V& t, V& sech2) {
  // |x| < 1/4: odd Taylor series x - x^3/3 + 2x^5/15 - 17x^7/315 + 62x^9/2835
  // (truncation < 3e-9 relative); else tanh|x| = (1 - e)/(1 + e), e = e^{-2|x|}
  // (1 - e >= 0.39 there, no cancellation).
  const V x2 = x * x;
  V q = vfma(x2, 62.f / 2835.f, -17.f / 315.f);
  q = vfma(q, x2, 2.f / 15.f);
  q = vfma(q, x2, -1.f / 3.f);
  q = vfma(q, x2, 1.f);
  const V ax = vabs(x);
  const V ex = vex2(ax * (-2.f * kLog2e));  // e^{-2|x|}
  const V inv = vrcp(1.f + ex);
  const V tl = vcopysign((1.f - ex) * inv, x);
  t = vsel(vlt(ax, 0.25f), x * q, tl);
  sech2 = 4.f * ex * (inv * inv);           // 1 - tanh^2 = 4 e/(1 + e)^2
}

// Weight activation for BF16-stored raw values by table: the entries hold vtanh of
// every BF16 magnitude in [2^-13, 64) (2432 values), formed on the device by vtanh
// itself, so there a lookup returns the bits of the evaluation. Outside, closed forms:
// from 64 on t = +-1 and 1 - tanh^2 = 0 (what vtanh gives there); below 2^-13 t = x
// (what the series gives) and 1 - tanh^2 = 1 (1 - x^2 rounded to FP32: x^2 < 2^-26 is
// under half the spacing of the floats below 1; vtanh's 4 e/(1 + e)^2 is within a
// few ulps of it). Layout: entry 0 the closed form below 2^-13, entries 1..2432 the
// magnitudes from 2^-13 up, entry 2433 the closed form from 64 on, so that an index is
// the magnitude bits clamped once on each side. An entry (A, B, C, 0) gives
// t = B x + copysign(A, x) and 1 - tanh^2 = C: (tanh|x_j|, 0, sech^2 x_j, 0) in the
// range, (1, 0, 0, 0) past it, (0, 1, 1, 0) below it. Finite inputs only (an infinite
// raw value gives NaN, where the evaluation gives +-1).
constexpr uint32_t kTanhLo = 0x3900u;                // BF16 magnitude bits of 2^-13
constexpr uint32_t kTanhHi = 0x4280u;                // BF16 magnitude bits of 64
constexpr uint32_t kTanhN = kTanhHi - kTanhLo;       // 2432 entries
constexpr uint32_t kTanhEntries = kTanhN + 2;        // and the two closed forms
constexpr uint32_t kTanhBytes = kTanhEntries * 16u;  // 38944 bytes of shared memory

// Fills the table (all threads of the block; the caller synchronises before use).
__device__ __forceinline__ void fill_tanh_table(float4* tab) {
  for (uint32_t j = threadIdx.x; j < kTanhEntries; j += blockDim.x) {
    float4 e;
    if (j == 0) {
      e = make_float4(0.f, 1.f, 1.f, 0.f);
    } else if (j <= kTanhN) {
      float t, s2;
      vtanh<float>(__uint_as_float((kTanhLo + j - 1u) << 16), t, s2);
      e = make_float4(t, 0.f, s2, 0.f);
    } else {
      e = make_float4(1.f, 0.f, 0.f, 0.f);
    }
    tab[j] = e;
  }
}

// tanh x and 1 - tanh^2 x for x a BF16 value (in an FP32 register) from the table.
__device__ __forceinline__ void tanh_lookup(const float4* tab, float x, float& t, float& sech2) {
  const uint32_t m = (__float_as_uint(x) >> 16) & 0x7fffu;
  const uint32_t j = min(max(m, kTanhLo - 1u) - (kTanhLo - 1u), kTanhN + 1u);
  const float4 e = tab[j];
  t = fmaf(e.y, x, copysignf(e.x, x));
  sech2 = e.z;
}
__device__ __forceinline__ void tanh_lookup(const float4* tab, P2 x, P2& t, P2& sech2) {
  tanh_lookup(tab, x.v.x, t.v.x, sech2.v.x);
  tanh_lookup(tab, x.v.y, t.v.y, sech2.v.y);
}

template <class V>
__device__ __forceinline__ V vlnkappa(V t, V kap) {
  const V s = t * vrcp(2.f + t);
  const V s2 = s * s;
  V q = vfma(s2, 1.f / 7.f, 1.f / 5.f);
  q = vfma(q, s2, 1.f / 3.f);
  q = vfma(q, s2, 1.f);
  const V ser = 2.f * s * q;
  const V lg = vlg2(kap) * kLn2;
  return vsel(vge(kap, 0.75f), ser, lg);
}

// Parity of the integer-valued float n.
__device__ __forceinline__ bool odd(float n) { return (static_cast<int>(n) & 1) != 0; }

__device__ __forceinline__ void carrier_fix(float n, float ps, float pc, float& h, float& s2x) {
  const bool o = odd(n);
  h = o ? ps * ps : pc * pc;
  const float sc = 2.f * ps * pc;
  s2x = o ? -sc : sc;
}
__device__ __forceinline__ void carrier_fix(P2 n, P2 ps, P2 pc, P2& h, P2& s2x) {
  carrier_fix(n.v.x, ps.v.x, pc.v.x, h.v.x, s2x.v.x);
  carrier_fix(n.v.y, ps.v.y, pc.v.y, h.v.y, s2x.v.y);
}

// The NASGabor carrier at x = k v / 2 (|x| <= 6400): h = cos^2 x = (1 + cos(k v))/2
// and sin 2x = sin(k v). With x = n pi/2 + r (Cody-Waite, pi/2 in three float
// parts, the first two with 12 significant bits so n*C1 and n*C2 are exact),
// cos^2 x is cos^2 r or sin^2 r by the parity of n, and sin 2x = (-1)^n 2 sin r cos r,
// with the Taylor polynomials of sin (to r^9) and cos (to r^10) on |r| <= pi/4.
template <class V>
__device__ __forceinline__ void vcarrier(V x, V& h, V& s2x) {
  constexpr float kTwoOverPi = 0.636619772367581343f;
  constexpr float kC1 = 1.5703125f;                // pi/2, first 12 bits
  constexpr float kC2 = 4.837512969970703125e-4f;  // next 12 bits
  constexpr float kC3 = 7.549790126404332e-8f;     // remainder
  const V n = vrint(x * kTwoOverPi);
  V r = vfma(n, -kC1, x);
  r = vfma(n, -kC2, r);
  r = vfma(n, -kC3, r);
  const V r2 = r * r;
  V ps = vfma(r2, kF9, -kF7);
  ps = vfma(ps, r2, kF5);
  ps = vfma(ps, r2, -kF3);
  ps = vfma(ps, r2, 1.f);
  ps = ps * r;
  V pc = vfma(r2, -1.f / 3628800.f, kF8);
  pc = vfma(pc, r2, -kF6);
  pc = vfma(pc, r2, kF4);
  pc = vfma(pc, r2, -kF2);
  pc = vfma(pc, r2, 1.f);
  carrier_fix(n, ps, pc, h, s2x);
}

// sin x and cos x (|x| <= 6400) from the same reduction, with the quadrant rotation.
__device__ __forceinline__ void quadrant(float n, float ps, float pc, float& s, float& c) {
  const int q = static_cast<int>(n) & 3;
  const float ss = (q & 1) ? pc : ps;
  const float cc = (q & 1) ? ps : pc;
  s = (q & 2) ? -ss : ss;
  c = ((q + 1) & 2) ? -cc : cc;
}

template <class V>
__device__ __forceinline__ void vsincos(V x, V& s, V& c);
template <>
__device__ __forceinline__ void vsincos<float>(float x, float& s, float& c) {
  constexpr float kTwoOverPi = 0.636619772367581343f;
  constexpr float kC1 = 1.5703125f;
  constexpr float kC2 = 4.837512969970703125e-4f;
  constexpr float kC3 = 7.549790126404332e-8f;
  const float n = rintf(x * kTwoOverPi);
  float r = fmaf(-n, kC1, x);
  r = fmaf(-n, kC2, r);
  r = fmaf(-n, kC3, r);
  const float r2 = r * r;
  float ps = fmaf(r2, kF9, -kF7);
  ps = fmaf(ps, r2, kF5);
  ps = fmaf(ps, r2, -kF3);
  ps = fmaf(ps, r2, 1.f);
  ps = ps * r;
  float pc = fmaf(r2, -1.f / 3628800.f, kF8);
  pc = fmaf(pc, r2, -kF6);
  pc = fmaf(pc, r2, kF4);
  pc = fmaf(pc, r2, -kF2);
  pc = fmaf(pc, r2, 1.f);
  quadrant(n, ps, pc, s, c);
}
template <>
__device__ __forceinline__ void vsincos<P2>(P2 x, P2& s, P2& c) {
  vsincos<float>(x.v.x, s.v.x, c.v.x);
  vsincos<float>(x.v.y, s.v.y, c.v.y);
}

// The phase-shifted carrier cos^2(y + w) and sin(2 (y + w)) for y = phi/2, w = k v/2,
// by angle addition from the sines and cosines of y and w. Summing y + w first would
// round w to the spacing of y (~1e-7 near pi/2), and near phi = pi, where cos(y + w)
// is itself ~k v, that rounding is most of the carrier.
template <class V>
__device__ __forceinline__ void vcarrier_sum(V y, V w, V& h, V& s2x) {
  V sy, cy, sw, cw;
  vsincos<V>(y, sy, cy);
  vsincos<V>(w, sw, cw);
  const V cx = vfma(cy, cw, -(sy * sw));
  const V sx = vfma(sy, cw, cy * sw);
  h = cx * cx;
  s2x = 2.f * sx * cx;
}

}  // namespace nasg
