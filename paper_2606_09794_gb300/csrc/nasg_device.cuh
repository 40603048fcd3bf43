// Device-side math of the NASGabor lobe (arXiv 2606.09794), shared by every
// NASGabor kernel of the library. FP32, generic over the value type V (one
// lobe as float, or two lobes packed as P2, see nasg_vec.cuh).
//
// The lobe (Sec. 5.1 definition, Supp. F factorisation):
//   u = d.z, v = d.x, kappa = (1+u)/2, tau = a v^2 / (1-u^2), E = kappa^tau,
//   p = exp(2 lam (E kappa - 1)), h = (1 + cos(k v))/2, G = C^-1 p E h,
//   C^-1 = lam sqrt(1+a) / (2 pi (1 - e^{-2 lam}))  (Supp. E/F; used for all Sec. 6 results),
//   or, with exact normalisation, 1 / (the Sec. 5.1 closed-form integral).
//
// FP32 formulation (algebraically identical, chosen for conditioning at lam
// up to 1e3, where 2 lam (E kappa - 1) amplifies any absolute error in 1 - u
// by 2 lam):
//   s2       = |d x z|^2                 (= 1 - u^2 without cancellation)
//   1 - u    = s2 / (1 + u) for u >= 0, else 1 - u   (and 1 + u symmetrically)
//   ln kappa = log1p(-(1 - u)/2) for u >= 0, log((1 + u)/2) for u < 0
//   E kappa - 1 = expm1((1 + tau) ln kappa)
//   p E      = exp(2 lam (E kappa - 1) + tau ln kappa)
//   h        = cos^2(k v / 2),  sin(k v) = 2 sin(k v/2) cos(k v/2)
//   1 - e^{-2 lam} = -expm1(-2 lam)
// Poles: where s2 == 0 in FP32 (below the normal range), u > 0 takes tau := 0
// (G = C^-1 h(v)) and u < 0 gives G := 0 with zero derivatives -- the same
// rule as the FP64 oracle.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nasg_fastmath.cuh"

namespace nasg {

constexpr float kInvTwoPi = 0.159154943091895336f;  // 1 / (2 pi)

// Lobe families (the NASGabor lobe and its specialisations; values equal the
// NASG_FAMILY_* codes of the C ABI):
//   NASGabor  G = C^-1 p E h               stored: lam, a, k, w
//   NASG      k = 0 (h = 1)                stored: lam, a, w
//   SG        a = 0, k = 0 (tau = 0, E = 1) stored: lam, w
//   phase     h = (1 + cos(k v + phi))/2    stored: lam, a, k, phi, w  (phi as is)
constexpr int kFamNasGabor = 0, kFamNasg = 1, kFamSg = 2, kFamPhase = 3;
template <int FAM>
struct Family {
  static constexpr bool HAS_A = FAM != kFamSg;
  static constexpr bool HAS_K = FAM == kFamNasGabor || FAM == kFamPhase;
  static constexpr bool HAS_PHASE = FAM == kFamPhase;
};
constexpr float kFltMin = 1.17549435e-38f;

// ---------------------------------------------------------------------------
// Loads of stored parameters
// ---------------------------------------------------------------------------

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ float to_float(float v) { return v; }
__device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }

// One element from GLOBAL memory (read-only path for f32); never use it on a
// shared-memory address.
template <typename T>
__device__ __forceinline__ float load1(const T* p);
template <>
__device__ __forceinline__ float load1<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load1<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(p[0]);
}

// Two consecutive elements (8 B f32 / 4 B bf16, aligned to that size).
template <typename T>
__device__ __forceinline__ P2 load2(const T* p);
template <>
__device__ __forceinline__ P2 load2<float>(const float* p) {
  P2 r;
  r.v = __ldg(reinterpret_cast<const float2*>(p));
  return r;
}
template <>
__device__ __forceinline__ P2 load2<__nv_bfloat16>(const __nv_bfloat16* p) {
  const uint32_t w = __ldg(reinterpret_cast<const unsigned int*>(p));
  return p2(bf16_lo(w), bf16_hi(w));
}

// ---------------------------------------------------------------------------
// Activations (Supp. C table) and their slopes d(activated)/d(raw)
// ---------------------------------------------------------------------------

template <class V>
struct Act {
  V lam, a, k, w[3];
  V s_lam, s_a, s_k, s_w[3];
  V phi;  // carrier phase (phase family; stored as is)
};

// r: lam_r, a_r, k_r, w_r, w_g, w_b. TAB: the raw values are BF16 and the weights'
// tanh comes from the block's table (tanh_lookup).
template <bool TAB = false, class V>
__device__ __forceinline__ void activate(const V* r, bool identity, Act<V>& o, const float4* tab = nullptr) {
  if (identity) {
    const V one = vconst<V>(1.f);
    o.lam = r[0]; o.a = r[1]; o.k = r[2];
    o.w[0] = r[3]; o.w[1] = r[4]; o.w[2] = r[5];
    o.s_lam = one; o.s_a = one; o.s_k = one;
    o.s_w[0] = one; o.s_w[1] = one; o.s_w[2] = one;
    return;
  }
  o.lam = vexp(r[0]);
  o.s_lam = o.lam;
  o.a = vexp(r[1]);
  o.s_a = o.a;
  // k = 20 (tanh r + 1) = 40 sig(2r); dk/dr = 20 (1 - tanh^2 r) = 80 sig (1 - sig).
  // Written through sig so that k keeps relative accuracy as tanh r -> -1.
  const V e = vexp(-2.f * r[2]);
  const V sig = vrcp(1.f + e);  // 0 when e overflows
  const V one_m_sig = vsel(vge(r[2], 0.f), e * sig, 1.f - sig);
  o.k = 40.f * sig;
  o.s_k = 80.f * sig * one_m_sig;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (TAB) {
      tanh_lookup(tab, r[3 + c], o.w[c], o.s_w[c]);
    } else {
      vtanh(r[3 + c], o.w[c], o.s_w[c]);
    }
  }
}

// Activations of a lobe family's stored scalars r = [lam, (a), (k), (phi), w_r, w_g, w_b];
// the quantities a family does not store are 0.
template <int FAM, class V>
__device__ __forceinline__ void activate_family(const V* r, bool identity, Act<V>& o) {
  using F = Family<FAM>;
  constexpr int A = 1, K = 1 + F::HAS_A, PH = K + F::HAS_K, W = PH + F::HAS_PHASE;
  const V zero = vconst<V>(0.f), one = vconst<V>(1.f);
  o.phi = F::HAS_PHASE ? r[PH] : zero;
  if (identity) {
    o.lam = r[0];
    o.a = F::HAS_A ? r[A] : zero;
    o.k = F::HAS_K ? r[K] : zero;
#pragma unroll
    for (int c = 0; c < 3; ++c) { o.w[c] = r[W + c]; o.s_w[c] = one; }
    o.s_lam = one; o.s_a = one; o.s_k = one;
    return;
  }
  o.lam = vexp(r[0]);
  o.s_lam = o.lam;
  o.a = zero; o.s_a = zero; o.k = zero; o.s_k = zero;
  if (F::HAS_A) {
    o.a = vexp(r[A]);
    o.s_a = o.a;
  }
  if (F::HAS_K) {
    const V e = vexp(-2.f * r[K]);
    const V sig = vrcp(1.f + e);
    const V one_m_sig = vsel(vge(r[K], 0.f), e * sig, 1.f - sig);
    o.k = 40.f * sig;
    o.s_k = 80.f * sig * one_m_sig;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) vtanh(r[W + c], o.w[c], o.s_w[c]);
}

// ---------------------------------------------------------------------------
// Frames: x and z axes of the lobe (y = z x x never formed; G does not use it)
// ---------------------------------------------------------------------------

template <class V>
struct QuatFrame {
  V q[4];       // raw quaternion (w, x, y, z)
  V inv2;       // 1/|q|^2
  V x[3], z[3];
};

// x = R(q/|q|) e_x, z = R(q/|q|) e_z from the homogeneous (degree-2) form of
// the rotation columns divided by |q|^2: an error in the computed 1/|q|^2 then
// only scales x and z, and the lobe math (1 - u from |d x z|^2) absorbs a
// scale, whereas the unit-quaternion form with an approximate q/|q| would
// rotate them slightly (which matters at sharpness ~1e3).
template <class V>
__device__ __forceinline__ void quat_frame(const V* qr, QuatFrame<V>& f) {
  const V qw = qr[0], qx = qr[1], qy = qr[2], qz = qr[3];
  const V ww = qw * qw, xx = qx * qx, yy = qy * qy, zz = qz * qz;
  const V n2 = (ww + xx) + (yy + zz);
  const V inv2 = vrcp(n2);
  f.inv2 = inv2;
  f.q[0] = qw; f.q[1] = qx; f.q[2] = qy; f.q[3] = qz;
  const V two_inv2 = 2.f * inv2;
  f.x[0] = ((ww + xx) - (yy + zz)) * inv2;
  f.x[1] = vfma(qx, qy, qw * qz) * two_inv2;
  f.x[2] = vfma(qx, qz, -(qw * qy)) * two_inv2;
  f.z[0] = vfma(qx, qz, qw * qy) * two_inv2;
  f.z[1] = vfma(qy, qz, -(qw * qx)) * two_inv2;
  f.z[2] = ((ww + zz) - (xx + yy)) * inv2;
}

// dLoss/dq_raw from dLoss/dx (L) and dLoss/dz (M). With x = x~(q)/|q|^2 and
// z = z~(q)/|q|^2 (x~, z~ quadratic in the raw quaternion q):
//   dLoss/dq_i = (2/|q|^2) [L.(dx~/dq_i)/2 + M.(dz~/dq_i)/2 - q_i (L.x + M.z)].
template <class V>
__device__ __forceinline__ void quat_frame_grad(const QuatFrame<V>& f, const V* L, const V* M, V* g) {
  const V w = f.q[0], x = f.q[1], y = f.q[2], z = f.q[3];
  const V s = vfma(L[0], f.x[0], vfma(L[1], f.x[1], vfma(L[2], f.x[2], vfma(M[0], f.z[0],
                  vfma(M[1], f.z[1], M[2] * f.z[2])))));
  const V k = 2.f * f.inv2;
  const V hw = vfma(L[0], w, vfma(L[1], z, vfma(M[0], y, vfma(M[2], w, -vfma(L[2], y, M[1] * x)))));
  const V hx = vfma(L[0], x, vfma(L[1], y, vfma(L[2], z, vfma(M[0], z, -vfma(M[1], w, M[2] * x)))));
  const V hy = vfma(L[1], x, vfma(M[0], w, vfma(M[1], z, -vfma(L[0], y, vfma(L[2], w, M[2] * y)))));
  const V hz = vfma(L[1], w, vfma(L[2], x, vfma(M[0], x, vfma(M[1], y, vfma(M[2], z, -(L[0] * z))))));
  g[0] = vfma(-w, s, hw) * k;
  g[1] = vfma(-x, s, hx) * k;
  g[2] = vfma(-y, s, hy) * k;
  g[3] = vfma(-z, s, hz) * k;
}

// dLoss/dq_raw for dLoss/dx = gv d and dLoss/dz = gu d (the lobe depends on the
// frame only through u = d.z and v = d.x). With x = x~(q)/|q|^2, z = z~(q)/|q|^2
// (x~, z~ quadratic in q):
//   dLoss/dq_i = (2/|q|^2) [gv d.(dx~/dq_i)/2 + gu d.(dz~/dq_i)/2 - q_i (gv v + gu u)],
// and the halved derivatives reduce to four combinations of d and q:
//   A1 = d0 w + d1 z - d2 y,  A2 = d0 x + d1 y + d2 z,  A3 = d0 y - d1 x + d2 w,
//   A4 = d0 z - d1 w - d2 x;
//   (w, x, y, z) components: gv A1 + gu A3, gv A2 + gu A4, gu A1 - gv A3, gu A2 - gv A4.
template <class V>
__device__ __forceinline__ void quat_frame_grad_d(const QuatFrame<V>& f, const V* d, V gv, V gu, V u, V v, V* g) {
  const V w = f.q[0], x = f.q[1], y = f.q[2], z = f.q[3];
  const V a1 = vfma(d[0], w, vfma(d[1], z, -(d[2] * y)));
  const V a2 = vfma(d[0], x, vfma(d[1], y, d[2] * z));
  const V a3 = vfma(d[0], y, vfma(d[2], w, -(d[1] * x)));
  const V a4 = vfma(d[0], z, -vfma(d[1], w, d[2] * x));
  const V s = vfma(gv, v, gu * u);
  const V k = 2.f * f.inv2;
  g[0] = vfma(-w, s, vfma(gv, a1, gu * a3)) * k;
  g[1] = vfma(-x, s, vfma(gv, a2, gu * a4)) * k;
  g[2] = vfma(-y, s, vfma(gu, a1, -(gv * a3))) * k;
  g[3] = vfma(-z, s, vfma(gu, a2, -(gv * a4))) * k;
}

// Supp. C frame from three cosines. RAW mode: c = tanh(r), s = sech(r) >= 0,
// with dc/dr = s^2 and ds/dr = -c s (finite everywhere, including where tanh
// saturates). IDENTITY mode: c = r, s = sqrt(1 - c^2), ds/dc = -c/s.
template <class V>
struct CosFrame {
  V c[3], s[3];     // cos / sin of theta, phi, psi
  V dc[3], ds[3];   // d c / d stored, d s / d stored
  V x[3], z[3];
};

template <class V>
__device__ __forceinline__ void cos_angle(V r, bool identity, V& c, V& s, V& dc, V& ds) {
  if (identity) {
    c = r;
    const V s2 = vmax((1.f - r) * (1.f + r), 0.f);
    const V rs = vrsqrt(vmax(s2, kFltMin));
    s = s2 * rs;
    dc = vconst<V>(1.f);
    ds = -(c * rs);
    return;
  }
  const V ar = vabs(r);
  const V em = vexp(-ar);                      // e^{-|r|}
  const V inv = vrcp(1.f + em * em);
  const V t = -(vexpm1n(-2.f * ar) * inv);     // tanh|r|
  c = vcopysign(t, r);
  s = 2.f * em * inv;                          // sech r
  dc = s * s;
  ds = -(c * s);
}

template <class V>
__device__ __forceinline__ void cos_frame(const V* r, bool identity, CosFrame<V>& f) {
  cos_angle(r[0], identity, f.c[0], f.s[0], f.dc[0], f.ds[0]);
  cos_angle(r[1], identity, f.c[1], f.s[1], f.dc[1], f.ds[1]);
  cos_angle(r[2], identity, f.c[2], f.s[2], f.dc[2], f.ds[2]);
  const V ct = f.c[0], st = f.s[0], cp = f.c[1], sp = f.s[1], cs = f.c[2], ss = f.s[2];
  f.z[0] = ct * sp; f.z[1] = st * sp; f.z[2] = cp;
  f.x[0] = vfma(ct * cp, cs, -(st * ss));
  f.x[1] = vfma(st * cp, cs, ct * ss);
  f.x[2] = -(sp * cs);
}

template <class V>
__device__ __forceinline__ void cos_frame_grad(const CosFrame<V>& f, const V* gx, const V* gz, V* g) {
  const V ct = f.c[0], st = f.s[0], cp = f.c[1], sp = f.s[1], cs = f.c[2], ss = f.s[2];
  const V g_ct = vfma(gx[0] * cp, cs, vfma(gx[1], ss, gz[0] * sp));
  const V g_st = vfma(gx[1] * cp, cs, vfma(gz[1], sp, -(gx[0] * ss)));
  const V g_cp = vfma(vfma(gx[0], ct, gx[1] * st), cs, gz[2]);
  const V g_sp = vfma(gz[0], ct, vfma(gz[1], st, -(gx[2] * cs)));
  const V g_cs = vfma(vfma(gx[0], ct, gx[1] * st), cp, -(gx[2] * sp));
  const V g_ss = vfma(gx[1], ct, -(gx[0] * st));
  g[0] = vfma(g_ct, f.dc[0], g_st * f.ds[0]);
  g[1] = vfma(g_cp, f.dc[1], g_sp * f.ds[1]);
  g[2] = vfma(g_cs, f.dc[2], g_ss * f.ds[2]);
}

// ---------------------------------------------------------------------------
// The lobe and its partial derivatives
// ---------------------------------------------------------------------------

// G_lam and G_a are the derivatives with respect to the stored scalars: dG/dlam and
// dG/da, or (logscale: raw activations, lam = e^{lam_r}, a = e^{a_r}) dG/dlam_r =
// lam dG/dlam and dG/da_r = a dG/da, which need no reciprocal of lam or 1 + a.
template <class V>
struct LobePartials {
  V G_u, G_v, G_lam, G_a, G_k;  // dG/du, dG/dv, dG/d(lam | lam_r), dG/d(a | a_r), dG/dk
  V G_phi;                      // dG/dphi (phase family)
  V u, v;                       // d.z and d.x
};

// ---------------------------------------------------------------------------
// Exact normalisation (Sec. 5.1 closed-form integral)
// ---------------------------------------------------------------------------
// 1 / int G = C^-1 R, with C^-1 the approximate constant and R = 2 / (1 + Psi):
//   Psi = 2 Lam e^{-Lam} S(sig) / (1 - e^{-2 Lam}),  Lam = lam (1 + a),  sig = Lam^2 - k^2,
//   S(sig) = sinh(sqrt sig)/sqrt sig, continued to sin(t)/t for sig = -t^2 (S is entire in sig).
// e^{-Lam} S and e^{-Lam} S' (S' = dS/dsig) are formed without overflow (Lam reaches 2e3):
//   |sig| <= 1: e^{-Lam} times the Taylor series of S and S' in sig (to sig^5);
//   sig > 1:    s = sqrt sig, A = e^{s - Lam} = e^{-k^2/(s + Lam)}, B = e^{-s - Lam},
//               e^{-Lam} S = (A - B)/(2 s),  e^{-Lam} S' = (s (A + B) - (A - B))/(4 s^3);
//   sig < -1:   t = sqrt(-sig) (t < k <= 40),  e^{-Lam} S = e^{-Lam} sin t / t,
//               e^{-Lam} S' = e^{-Lam} (sin t - t cos t)/(2 t^3).
// Psi > -0.22 everywhere (Lam e^{-Lam} / (1 - e^{-2 Lam}) <= 1/2 and sin t / t >= -0.22).
// Derivatives: d ln R = -(R/2) dPsi with
//   dPsi/dk   = -2 k c e^{-Lam} S',  c = 2 Lam / (1 - e^{-2 Lam}),
//   dPsi/dLam = Psi (1/Lam - coth Lam) + 2 Lam c e^{-Lam} S',
// where for sig > 1 the second form is rearranged so that no two large terms cancel
// (they do when Lam >> k, where dPsi/dLam ~ k^2 / (2 Lam^2)):
//   dPsi/dLam = -Psi (k^2 / (Lam s^2) + 2 e^{-2 Lam}/(1 - e^{-2 Lam}))
//               + Lam (A k^2 / (s + Lam) + B (s + Lam)) / (s^2 (1 - e^{-2 Lam})),
// and 1/Lam - coth Lam = -(Lam/3 - Lam^3/45 + 2 Lam^5/945 - Lam^7/4725 + 2 Lam^9/93555)
// below Lam = 1/2. dLam/dlam = 1 + a, dLam/da = lam.
// With a carrier phase phi the sin(k v) sin(phi) part of the carrier integrates
// to zero (the envelope is even in v), so R = 2 / (1 + cos(phi) Psi), its
// Lam / k derivatives scale by cos(phi), and d ln R/dphi = (R/2) sin(phi) Psi.
// 1 + cos(phi) Psi cancels where phi ~ pi and Psi ~ 1 (k << Lam: the lobe's integral
// tends to 0), so it is formed as (1 - Psi) + 2 cos^2(phi/2) Psi with 1 - Psi from
// its own expression: for sig > 1, with delta = k^2/(s + Lam) = Lam - s and
// e^{-delta} - 1 = em,
//   (1 - Psi)(1 - e^{-2 Lam}) = -em - (delta/s)(1 + em) + e^{-2 Lam} (delta/s - em) / (1 + em);
// for |sig| <= 1 and Lam <= 1, from S(Lam^2) c e^{-Lam} = 1 (the k = 0 integral),
//   1 - Psi = c e^{-Lam} (S(Lam^2) - S(sig)) = c e^{-Lam} k^2 sum_n D_n/(2n+1)!,
//   D_1 = 1, D_{n+1} = Lam^2 D_n + sig^n (the difference quotient of x^n);
// elsewhere Psi < 0.9 and 1 - Psi has no cancellation. Where R is that large its
// derivative needs dPsi/dLam to full relative accuracy too (it is O(k^2) while its
// usual form is a difference of O(Lam) terms), so the phase path forms it as
//   sig > 1:  d ln Psi/dLam = -k^2/(Lam s^2) + (delta/s) coth s + sinh delta/(sinh s sinh Lam),
//             the last term 2 e^{-2s} (1 - e^{-2 delta}) / ((1 - e^{-2s})(1 - e^{-2 Lam}));
//   |sig| <= 1, Lam <= 1, from Psi = S(sig)/S(Lam^2):
//             dPsi/dLam = (2 Lam / S(Lam^2)) (-k^2 sum_m (m+1) D_m/(2m+3)! + (1 - Psi) S'(Lam^2)).
template <bool GRAD, bool PHASE = false>
__device__ __forceinline__ void exact_norm1(float lam, float a, float k, float& r, float& dl, float& da,
                                            float& dk, float phi = 0.f, float* dphi = nullptr) {
  const float opa = 1.f + a;
  const float L = lam * opa;
  const float sig = (L - k) * (L + k);
  const float om = -vexpm1n(-2.f * L);  // 1 - e^{-2 Lam}
  const float rom = rcpa(om);
  const float c = 2.f * L * rom;
  float es, esp, dpsi_dl = 0.f;
  bool rearranged = false;
  float s = 0.f, A = 0.f, B = 0.f, rs2 = 0.f;
  float omp = 0.f;        // 1 - Psi where it needs its own expression (PHASE)
  bool have_omp = false;
  float dpsi_acc = 0.f;   // dPsi/dLam in full relative accuracy (PHASE, same branches)
  if (fabsf(sig) <= 1.f) {
    const float el = vexp(-L);
    if (PHASE && L <= 1.f) {
      const float L2 = L * L;
      // 1/(2n+1)! for n = 1..6
      const float inv_fact[6] = {1.f / 6.f, 1.f / 120.f, 1.f / 5040.f, 1.f / 362880.f, 1.f / 39916800.f,
                                 1.f / 6227020800.f};
      float dn = 1.f, pw = sig, acc = 0.f, acc2 = 0.f;
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        acc = fmaf(dn, inv_fact[j], acc);
        acc2 = fmaf(float(j + 2) * dn, inv_fact[j + 1], acc2);
        dn = fmaf(L2, dn, pw);
        pw *= sig;
      }
      const float ce = c * el;  // = 1/S(Lam^2)
      omp = ce * (k * k) * acc;
      have_omp = true;
      // S'(Lam^2) by its series (the coefficients of Sp below)
      float spx = fmaf(L2, 1.f / 1037836800.f, 1.f / 7983360.f);
      spx = fmaf(spx, L2, 1.f / 90720.f);
      spx = fmaf(spx, L2, 1.f / 1680.f);
      spx = fmaf(spx, L2, 1.f / 60.f);
      spx = fmaf(spx, L2, 1.f / 6.f);
      dpsi_acc = 2.f * L * ce * fmaf(omp, spx, -(k * k) * acc2);
    }
    float S = fmaf(sig, 1.f / 39916800.f, 1.f / 362880.f);
    S = fmaf(S, sig, 1.f / 5040.f);
    S = fmaf(S, sig, 1.f / 120.f);
    S = fmaf(S, sig, 1.f / 6.f);
    S = fmaf(S, sig, 1.f);
    float Sp = fmaf(sig, 1.f / 1037836800.f, 1.f / 7983360.f);
    Sp = fmaf(Sp, sig, 1.f / 90720.f);
    Sp = fmaf(Sp, sig, 1.f / 1680.f);
    Sp = fmaf(Sp, sig, 1.f / 60.f);
    Sp = fmaf(Sp, sig, 1.f / 6.f);
    es = el * S;
    esp = el * Sp;
  } else if (sig > 0.f) {
    const float rs = rsqa(sig);
    s = sig * rs;
    rs2 = rs * rs;
    A = vexp(-(k * k) * rcpa(s + L));
    B = vexp(-s - L);
    es = (A - B) * (0.5f * rs);
    esp = fmaf(s, A + B, B - A) * (0.25f * rs2 * rs);
    rearranged = true;
    if (PHASE) {
      const float delta = (k * k) * rcpa(s + L);
      const float em = vexpm1n(-delta);
      const float q = delta * rs;
      omp = (-em - q * (1.f + em) + vexp(-2.f * L) * (q - em) * rcpa(1.f + em)) * rom;
      have_omp = true;
      if (GRAD) {
        const float e2s = vexp(-2.f * s);
        const float roms = rcpa(-vexpm1n(-2.f * s));  // 1/(1 - e^{-2s})
        const float t1 = -(k * k) * rcpa(L) * rs2;
        const float t2 = q * (1.f + e2s) * roms;
        const float t3 = -2.f * e2s * vexpm1n(-2.f * delta) * roms * rom;
        dpsi_acc = (c * es) * (t1 + t2 + t3);
      }
    }
  } else {
    const float rt = rsqa(-sig);
    const float t = -sig * rt;
    float sn, cs;
    vsincos<float>(t, sn, cs);
    const float el = vexp(-L);
    es = el * sn * rt;
    esp = el * fmaf(-t, cs, sn) * (0.5f * rt * rt * rt);
  }
  const float psi = c * es;
  float cph = 1.f, sph = 0.f;
  if (PHASE) {
    vsincos<float>(phi, sph, cph);
    float sh, ch;  // 1 + cos(phi) = 2 cos^2(phi/2)
    vsincos<float>(0.5f * phi, sh, ch);
    r = 2.f * rcpa(fmaf(2.f * ch * ch, psi, have_omp ? omp : 1.f - psi));
  } else {
    r = 2.f * rcpa(1.f + psi);
  }
  if (GRAD) {
    if (rearranged) {
      const float e2 = vexp(-2.f * L);
      const float kk = k * k;
      const float pos = L * fmaf(A * kk, rcpa(s + L), B * (s + L)) * rs2 * rom;
      dpsi_dl = fmaf(-psi, fmaf(kk * rcpa(L), rs2, 2.f * e2 * rom), pos);
    } else {
      float lg;  // 1/Lam - coth Lam
      if (L < 0.5f) {
        const float x2 = L * L;
        float q = fmaf(x2, 2.f / 93555.f, -1.f / 4725.f);
        q = fmaf(q, x2, 2.f / 945.f);
        q = fmaf(q, x2, -1.f / 45.f);
        q = fmaf(q, x2, 1.f / 3.f);
        lg = -L * q;
      } else {
        lg = rcpa(L) - fmaf(2.f, rom, -1.f);
      }
      dpsi_dl = fmaf(psi, lg, 2.f * L * c * esp);
    }
    if (PHASE && have_omp) dpsi_dl = dpsi_acc;
    const float dpsi_dk = -2.f * k * c * esp;
    const float h = -0.5f * r * cph;
    dl = h * dpsi_dl * opa;
    da = h * dpsi_dl * lam;
    dk = h * dpsi_dk;
    if (PHASE) *dphi = 0.5f * r * sph * psi;
  }
}

template <bool GRAD>
__device__ __forceinline__ void exact_norm(float lam, float a, float k, float& r, float& dl, float& da, float& dk) {
  exact_norm1<GRAD>(lam, a, k, r, dl, da, dk);
}
template <bool GRAD>
__device__ __forceinline__ void exact_norm(P2 lam, P2 a, P2 k, P2& r, P2& dl, P2& da, P2& dk) {
  exact_norm1<GRAD>(lam.v.x, a.v.x, k.v.x, r.v.x, dl.v.x, da.v.x, dk.v.x);
  exact_norm1<GRAD>(lam.v.y, a.v.y, k.v.y, r.v.y, dl.v.y, da.v.y, dk.v.y);
}
template <bool GRAD>
__device__ __forceinline__ void exact_norm_phase(float lam, float a, float k, float phi, float& r, float& dl,
                                                 float& da, float& dk, float& dphi) {
  exact_norm1<GRAD, true>(lam, a, k, r, dl, da, dk, phi, &dphi);
}
template <bool GRAD>
__device__ __forceinline__ void exact_norm_phase(P2 lam, P2 a, P2 k, P2 phi, P2& r, P2& dl, P2& da, P2& dk,
                                                 P2& dphi) {
  exact_norm1<GRAD, true>(lam.v.x, a.v.x, k.v.x, r.v.x, dl.v.x, da.v.x, dk.v.x, phi.v.x, &dphi.v.x);
  exact_norm1<GRAD, true>(lam.v.y, a.v.y, k.v.y, r.v.y, dl.v.y, da.v.y, dk.v.y, phi.v.y, &dphi.v.y);
}

// The direction-independent factors of one lobe: the normalisation C^-1 (approximate,
// or exact with the Sec. 5.1 closed form) and its logarithmic derivatives. A kernel that
// evaluates a lobe at many directions forms them once (lobe_norm) and evaluates each
// direction with lobe_at; lobe_family does both for one direction.
template <class V>
struct LobeNorm {
  V cinv, dlam, da, dk, dphi;  // C^-1 and d ln C^-1 / d(lam | lam_r, a | a_r, k, phi) (see LobePartials)
};

template <bool GRAD, int FAM, class V>
__device__ __forceinline__ void lobe_norm(V lam, V a, V k, V phi, bool normalised, bool exact, bool logscale,
                                          LobeNorm<V>& nc) {
  using F = Family<FAM>;
  nc.cinv = vconst<V>(1.f);
  nc.dlam = vconst<V>(0.f);
  nc.da = vconst<V>(0.f);
  nc.dk = vconst<V>(0.f);
  nc.dphi = vconst<V>(0.f);
  if (!normalised) return;
  const V em = vexpm1n(-2.f * lam);  // e^{-2 lam} - 1 (negative)
  const V r_em = vrcp(em);
  V rs = vconst<V>(1.f);  // 1/sqrt(1 + a)
  if (F::HAS_A) {
    const V opa = 1.f + a;
    rs = vrsqrt(opa);
    nc.cinv = -((lam * (opa * rs)) * (kInvTwoPi * r_em));
  } else {
    nc.cinv = -(lam * (kInvTwoPi * r_em));
  }
  if (GRAD) {
    // d ln C^-1/d lam = 1/lam - 2 e^{-2 lam}/(1 - e^{-2 lam}); d ln C^-1/d a = 1/(2 (1+a));
    // logscale: lam d ln C^-1/d lam = 1 + 2 lam (1 + em)/em, a d ln C^-1/d a = a rs^2 / 2
    if (logscale) {
      nc.dlam = vfma(2.f * lam * (1.f + em), r_em, 1.f);
      if (F::HAS_A) nc.da = 0.5f * a * (rs * rs);
    } else {
      nc.dlam = vfma(2.f * (1.f + em), r_em, vrcp(lam));
      if (F::HAS_A) nc.da = 0.5f * (rs * rs);
    }
  }
  // without a carrier the closed form is the NASG constant itself (Psi = 1)
  if (exact && F::HAS_PHASE) {
    V r, dr_lam, dr_a, dr_k, dr_phi;
    exact_norm_phase<GRAD>(lam, a, k, phi, r, dr_lam, dr_a, dr_k, dr_phi);
    nc.cinv = nc.cinv * r;
    if (GRAD) {
      nc.dlam = logscale ? vfma(lam, dr_lam, nc.dlam) : nc.dlam + dr_lam;
      nc.da = logscale ? vfma(a, dr_a, nc.da) : nc.da + dr_a;
      nc.dk = dr_k;
      nc.dphi = dr_phi;
    }
  } else if (exact && F::HAS_K) {
    V r, dr_lam, dr_a, dr_k;
    exact_norm<GRAD>(lam, a, k, r, dr_lam, dr_a, dr_k);
    nc.cinv = nc.cinv * r;
    if (GRAD) {
      nc.dlam = logscale ? vfma(lam, dr_lam, nc.dlam) : nc.dlam + dr_lam;
      nc.da = logscale ? vfma(a, dr_a, nc.da) : nc.da + dr_a;
      nc.dk = dr_k;
    }
  }
}

// One lobe of family FAM at direction d, given its normalisation factors nc (a, k,
// phi ignored where the family has none; see Family). PER_G: G_u, G_a and G_lam are
// returned divided by G (the caller multiplies them by G once, with its upstream factor).
template <bool GRAD, int FAM, class V, bool PER_G = false>
__device__ __forceinline__ V lobe_at(const V* d, const V* x, const V* z, V lam, V a, V k, V phi,
                                     const LobeNorm<V>& nc, bool exact, bool logscale, LobePartials<V>* pd) {
  using F = Family<FAM>;
  using M = typename VecTraits<V>::Mask;
  const V u = vfma(d[0], z[0], vfma(d[1], z[1], d[2] * z[2]));
  const V v = vfma(d[0], x[0], vfma(d[1], x[1], d[2] * x[2]));
  const V cx = vfma(d[1], z[2], -(d[2] * z[1]));
  const V cy = vfma(d[2], z[0], -(d[0] * z[2]));
  const V cz = vfma(d[0], z[1], -(d[1] * z[0]));
  const V s2 = vfma(cx, cx, vfma(cy, cy, cz * cz));  // 1 - u^2
  // pole: s2 below the normal range (the FP32 zero of 1 - u^2)
  const M pole = vlt(s2, kFltMin);
  const M up = vge(u, 0.f);
  const M anti = vand(pole, vnot(up));
  const V inv_s2 = vsel(pole, 0.f, vrcp(s2));
  // 1 - u and 1 + u, each from s2 on the side where it is small
  V t, kap, inv_opu;
  if constexpr (F::HAS_A) {
    // 1 + |u| and 1 - |u| = s2/(1 + |u|); t = kappa - 1 = -(1 - u)/2 is only read where
    // kappa >= 3/4 (the series of ln kappa), i.e. where u > 0 and 1 - u = 1 - |u|
    const V big = 1.f + vabs(u);
    const V rb = vrcp(big);
    const V small = s2 * rb;
    const V opu = vsel(up, big, small);
    inv_opu = vsel(up, rb, big * inv_s2);  // 1/(1+u) = 1/(2 kappa)
    t = -0.5f * small;
    kap = 0.5f * opu;
  } else {
    const V one_m_u = 1.f - u, one_p_u = 1.f + u;
    const V rd = vrcp(vsel(up, one_p_u, one_m_u));
    const V omu = vsel(up, s2 * rd, one_m_u);
    const V opu = vsel(up, one_p_u, s2 * rd);
    inv_opu = vsel(up, rd, one_m_u * inv_s2);
    t = -0.5f * omu;
    kap = vsel(up, 1.f + t, 0.5f * opu);
  }
  // without anisotropy (SG): tau = 0, E = 1, E kappa - 1 = kappa - 1 = t exactly
  const V ln_k = F::HAS_A ? vsel(anti, 0.f, vlnkappa(t, vmax(kap, kFltMin))) : vconst<V>(0.f);  // ln kappa
  const V tau = F::HAS_A ? a * v * v * inv_s2 : vconst<V>(0.f);
  const V ln_e = tau * ln_k;                                      // ln E
  // E kappa - 1 and E kappa, each to full relative accuracy (E kappa is tiny far from the
  // lobe, where 2 lam E kappa / (1 + u) = lam E still enters dG/du)
  V em1, ek;
  if (F::HAS_A) {
    vexp_expm1n(ln_e + ln_k, ek, em1);
  } else {
    em1 = t;    // kappa - 1
    ek = kap;   // kappa
  }
  const V two_lam = 2.f * lam;
  const V pe = F::HAS_A ? vexp(vfma(two_lam, em1, ln_e)) : vexp(two_lam * t);  // p E
  V h = vconst<V>(1.f), sin_kv = vconst<V>(0.f);  // (1 + cos(k v + phi))/2 and sin(k v + phi)
  if (F::HAS_PHASE) {
    vcarrier_sum(0.5f * phi, 0.5f * k * v, h, sin_kv);
  } else if (F::HAS_K) {
    vcarrier(0.5f * k * v, h, sin_kv);
  }
  // the antipode (G := 0 with zero derivatives) is applied once, through C^-1 p E;
  // every other factor below is finite there (tau, ln kappa, 1/(1+u) are 0)
  const V cpe = vsel(anti, 0.f, nc.cinv * pe);
  const V G = cpe * h;
  if (GRAD) {
    pd->u = u;
    pd->v = v;
    const V two_lam_ek = two_lam * ek;
    const V dtau_du = 2.f * u * tau * inv_s2;
    const V dtau_dv = 2.f * a * v * inv_s2;
    const V dlne_du = vfma(ln_k, dtau_du, tau * inv_opu);
    const V dlne_dv = ln_k * dtau_dv;
    const V cpe_sin = cpe * sin_kv;                     // C^-1 p E sin(k v + phi)
    if (F::HAS_A) {
      const V f_u = vfma(two_lam_ek, dlne_du + inv_opu, dlne_du);
      pd->G_u = PER_G ? f_u : G * f_u;
      const V gv_env = G * (two_lam_ek + 1.f) * dlne_dv;
      pd->G_v = F::HAS_K ? vfma(G * (two_lam_ek + 1.f), dlne_dv, -(cpe_sin * (0.5f * k))) : gv_env;
      // d(tau)/da = v^2/(1-u^2); logscale: a d(tau)/da = tau
      const V f_a = vfma((two_lam_ek + 1.f) * ln_k, logscale ? tau : v * v * inv_s2, nc.da);
      pd->G_a = PER_G ? f_a : G * f_a;
    } else {
      pd->G_u = PER_G ? lam : G * lam;                  // d/du 2 lam (kappa - 1) = lam
      pd->G_v = vconst<V>(0.f);
      pd->G_a = vconst<V>(0.f);
    }
    if (F::HAS_K) {
      pd->G_k = exact ? vfma(G, nc.dk, -(cpe_sin * (0.5f * v))) : -(cpe_sin * (0.5f * v));
    } else {
      pd->G_k = vconst<V>(0.f);
    }
    pd->G_phi = F::HAS_PHASE ? (exact ? vfma(G, nc.dphi, -(0.5f * cpe_sin)) : -(0.5f * cpe_sin))
                             : vconst<V>(0.f);
    const V f_lam = vfma(logscale ? two_lam : vconst<V>(2.f), em1, nc.dlam);
    pd->G_lam = PER_G ? f_lam : G * f_lam;
  }
  return G;
}

// One lobe of family FAM at one direction (normalisation included).
template <bool GRAD, int FAM, class V>
__device__ __forceinline__ V lobe_family(const V* d, const V* x, const V* z, V lam, V a, V k, V phi,
                                         bool normalised, bool exact, bool logscale, LobePartials<V>* pd) {
  LobeNorm<V> nc;
  lobe_norm<GRAD, FAM>(lam, a, k, phi, normalised, exact, logscale, nc);
  return lobe_at<GRAD, FAM>(d, x, z, lam, a, k, phi, nc, exact, logscale, pd);
}

// The NASGabor lobe.
template <bool GRAD, class V>
__device__ __forceinline__ V lobe(const V* d, const V* x, const V* z, V lam, V a, V k, bool normalised, bool exact,
                                  bool logscale, LobePartials<V>* pd) {
  return lobe_family<GRAD, kFamNasGabor>(d, x, z, lam, a, k, vconst<V>(0.f), normalised, exact, logscale, pd);
}

// ---------------------------------------------------------------------------
// View direction d = (mu - cam)/|mu - cam|
// ---------------------------------------------------------------------------

__device__ __forceinline__ float view_dir(const float* means, int64_t i, float cx, float cy, float cz,
                                          float d[3]) {
  const float rx = __ldg(means + 3 * i + 0) - cx;
  const float ry = __ldg(means + 3 * i + 1) - cy;
  const float rz = __ldg(means + 3 * i + 2) - cz;
  const float inv = rsqrtf(rx * rx + ry * ry + rz * rz);
  d[0] = rx * inv; d[1] = ry * inv; d[2] = rz * inv;
  return inv;
}

// The per-primitive scalar arithmetic of the kernels (view direction, dot products,
// dLoss/dmu) with every operation explicitly rounded, so that no contraction choice is
// left to the compiler and every kernel instance forms the same bits for the same inputs.
__device__ __forceinline__ float view_dir_rn(const float mu[3], const float cam[3], float d[3]) {
  const float rx = __fsub_rn(mu[0], cam[0]), ry = __fsub_rn(mu[1], cam[1]), rz = __fsub_rn(mu[2], cam[2]);
  const float inv = rsqrtf(__fmaf_rn(rz, rz, __fmaf_rn(ry, ry, __fmul_rn(rx, rx))));
  d[0] = __fmul_rn(rx, inv);
  d[1] = __fmul_rn(ry, inv);
  d[2] = __fmul_rn(rz, inv);
  return inv;
}
__device__ __forceinline__ float dot3_rn(const float a[3], const float b[3]) {
  return __fmaf_rn(a[2], b[2], __fmaf_rn(a[1], b[1], __fmul_rn(a[0], b[0])));
}
// component c of dLoss/dmu = (gd_c - (gd . d) d_c) / |mu - cam|
__device__ __forceinline__ float mean_grad_rn(float gd_c, float dot, float d_c, float inv_dist) {
  return __fmul_rn(__fmaf_rn(-dot, d_c, gd_c), inv_dist);
}

// dLoss/dmu = (I - d d^T) dLoss/dd / |mu - cam|
__device__ __forceinline__ void dir_grad(const float d[3], const float gd[3], float inv_dist, float gm[3]) {
  const float dot = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
  gm[0] = (gd[0] - dot * d[0]) * inv_dist;
  gm[1] = (gd[1] - dot * d[1]) * inv_dist;
  gm[2] = (gd[2] - dot * d[2]) * inv_dist;
}

}  // namespace nasg
