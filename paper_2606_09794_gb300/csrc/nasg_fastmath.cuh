// FP32 elementary functions for the NASGabor kernels, generic over the value
// type V (float, or the packed pair P2 of nasg_vec.cuh), written from their
// series definitions and the hardware ex2/lg2/rcp approximations (no vendor
// math code). Each is checked on the GPU against float64 references through
// the library's math probe (tests/test_gpu_math.py).
//
//   vexp(x)       2^(x log2 e) by ex2.approx (relative error ~2^-22 plus the
//                 rounding of x log2 e, i.e. ~|x| 6e-8).
//   vexpm1n(y)    e^y - 1 for y <= 0: Taylor polynomial to y^9 on [-0.5, 0]
//                 (truncation < 3e-10 relative), 2^(y log2 e) - 1 below -0.5
//                 (|result| >= 0.39 there, so the subtraction loses nothing).
//   vtanh(x)      e = e^{-2|x|} - 1, tanh|x| = -e/(2 + e), and
//                 1 - tanh^2 x = 4 e^{-2|x|}/(2 + e)^2 without cancellation.
//   vlnkappa(t)   ln(1 + t) for t in [-1, 0]: 2 atanh(t/(2 + t)) series to
//                 s^9 where 1 + t >= 0.75, lg2.approx elsewhere.
//   vsincos(x)    |x| <= 6400: Cody-Waite reduction x = n pi/2 + r with pi/2
//                 split in three float parts (the first two with 12
//                 significant bits, so n*C1 and n*C2 are exact), Taylor
//                 polynomials of sin (to r^9) and cos (to r^10) on
//                 |r| <= pi/4 (truncation < 3e-9), then the quadrant rotation.
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
  V p = vfma(y, kF9, kF8);
  p = vfma(p, y, kF7);
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

template <class V>
__device__ __forceinline__ void vtanh(V x, V& t, V& sech2) {
  const V y = -2.f * vabs(x);
  const V ex = vex2(y * kLog2e);                        // e^{-2|x|}
  const V e = vsel(vgt(y, -0.5f), taylor_expm1(y), ex - 1.f);  // e^{-2|x|} - 1
  const V inv = vrcp(2.f + e);
  t = vcopysign(-e * inv, x);
  sech2 = 4.f * ex * inv * inv;
}

template <class V>
__device__ __forceinline__ V vlnkappa(V t, V kap) {
  const V s = t * vrcp(2.f + t);
  const V s2 = s * s;
  V q = vfma(s2, 1.f / 9.f, 1.f / 7.f);
  q = vfma(q, s2, 1.f / 5.f);
  q = vfma(q, s2, 1.f / 3.f);
  q = vfma(q, s2, 1.f);
  const V ser = 2.f * s * q;
  const V lg = vlg2(kap) * kLn2;
  return vsel(vge(kap, 0.75f), ser, lg);
}

__device__ __forceinline__ void quadrant(float n, float ps, float pc, float& s, float& c) {
  const int q = static_cast<int>(n) & 3;
  const float ss = (q & 1) ? pc : ps;
  const float cc = (q & 1) ? ps : pc;
  s = (q & 2) ? -ss : ss;
  c = ((q + 1) & 2) ? -cc : cc;
}
__device__ __forceinline__ void quadrant(P2 n, P2 ps, P2 pc, P2& s, P2& c) {
  quadrant(n.v.x, ps.v.x, pc.v.x, s.v.x, c.v.x);
  quadrant(n.v.y, ps.v.y, pc.v.y, s.v.y, c.v.y);
}

template <class V>
__device__ __forceinline__ void vsincos(V x, V& s, V& c) {
  constexpr float kTwoOverPi = 0.636619772367581343f;
  constexpr float kC1 = 1.5703125f;                // pi/2, first 12 bits
  constexpr float kC2 = 4.837512969970703125e-4f;  // next 12 bits
  constexpr float kC3 = 7.549790126404332e-8f;     // remainder
  const V n = vrint(x * kTwoOverPi);
  V r = vfma(n, -kC1, x);
  r = vfma(n, -kC2, r);
  r = vfma(n, -kC3, r);
  const V r2 = r * r;
  // sin r = r (1 - r^2/3! + r^4/5! - r^6/7! + r^8/9!)
  V ps = vfma(r2, kF9, -kF7);
  ps = vfma(ps, r2, kF5);
  ps = vfma(ps, r2, -kF3);
  ps = vfma(ps, r2, 1.f);
  ps = ps * r;
  // cos r = 1 - r^2/2! + r^4/4! - r^6/6! + r^8/8! - r^10/10!
  V pc = vfma(r2, -1.f / 3628800.f, kF8);
  pc = vfma(pc, r2, -kF6);
  pc = vfma(pc, r2, kF4);
  pc = vfma(pc, r2, -kF2);
  pc = vfma(pc, r2, 1.f);
  quadrant(n, ps, pc, s, c);
}

}  // namespace nasg
