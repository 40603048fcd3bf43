// Device-side math of the NASGabor lobe (arXiv 2606.09794), shared by every
// NASGabor kernel of the library. FP32 throughout.
//
// The lobe (Sec. 4.1 definition, Supp. F factorisation):
//   u = d.z, v = d.x, kappa = (1+u)/2, tau = a v^2 / (1-u^2), E = kappa^tau,
//   p = exp(2 lam (E kappa - 1)), h = (1 + cos(k v))/2, G = C^-1 p E h,
//   C^-1 = lam sqrt(1+a) / (2 pi (1 - e^{-2 lam}))  (Supp. E/F; used for all Sec. 5 results).
//
// FP32 formulation (algebraically identical, chosen for conditioning at
// lam up to 1e3, where 2 lam (E kappa - 1) amplifies any absolute error in
// 1 - u by 2 lam):
//   s2      = |d x z|^2                 (= 1 - u^2 without cancellation)
//   1 - u   = s2 / (1 + u) for u >= 0, else 1 - u
//   ln kappa = log1p(-(1 - u)/2)
//   E kappa - 1 = expm1((1 + tau) ln kappa)
//   p E     = exp(2 lam (E kappa - 1) + tau ln kappa)
//   h       = cos^2(k v / 2),  sin(k v) = 2 sin(k v/2) cos(k v/2)
//   1 - e^{-2 lam} = -expm1(-2 lam)
// Poles: where s2 == 0, u > 0 takes tau := 0 (G = C^-1 h(v)) and u < 0 gives
// G := 0 with zero derivatives -- the same rule as the FP64 oracle.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace nasg {

constexpr float kInvTwoPi = 0.159154943091895336f;  // 1 / (2 pi)

// ---------------------------------------------------------------------------
// Loads of stored parameters
// ---------------------------------------------------------------------------

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// Load V consecutive elements starting at p (V = 1 or 4; V = 4 requires
// 16-byte alignment for float and 8-byte alignment for bfloat16).
template <typename T, int V>
struct VecLoad;

template <>
struct VecLoad<float, 1> {
  static __device__ __forceinline__ void run(const float* p, float* o) { o[0] = __ldg(p); }
};
template <>
struct VecLoad<float, 4> {
  static __device__ __forceinline__ void run(const float* p, float* o) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  }
};
template <>
struct VecLoad<__nv_bfloat16, 1> {
  static __device__ __forceinline__ void run(const __nv_bfloat16* p, float* o) {
    o[0] = __bfloat162float(p[0]);
  }
};
template <>
struct VecLoad<__nv_bfloat16, 4> {
  static __device__ __forceinline__ void run(const __nv_bfloat16* p, float* o) {
    uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    o[0] = bf16_lo(t.x); o[1] = bf16_hi(t.x); o[2] = bf16_lo(t.y); o[3] = bf16_hi(t.y);
  }
};

template <int V>
struct VecStore;
template <>
struct VecStore<1> {
  static __device__ __forceinline__ void run(float* p, const float* v, bool acc) {
    p[0] = acc ? p[0] + v[0] : v[0];
  }
};
template <>
struct VecStore<4> {
  static __device__ __forceinline__ void run(float* p, const float* v, bool acc) {
    float4* q = reinterpret_cast<float4*>(p);
    float4 t = make_float4(v[0], v[1], v[2], v[3]);
    if (acc) {
      float4 o = *q;
      t.x += o.x; t.y += o.y; t.z += o.z; t.w += o.w;
    }
    *q = t;
  }
};

template <typename T>
__device__ __forceinline__ float load1(const T* p);
template <>
__device__ __forceinline__ float load1<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load1<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(p[0]);
}

// ---------------------------------------------------------------------------
// Activations (Supp. C table) and their slopes d(activated)/d(raw)
// ---------------------------------------------------------------------------

struct Act {
  float lam, a, k, w[3];
  float s_lam, s_a, s_k, s_w[3];
};

__device__ __forceinline__ void activate(float lam_r, float a_r, float k_r, float w0, float w1,
                                         float w2, bool identity, Act& o) {
  if (identity) {
    o.lam = lam_r; o.a = a_r; o.k = k_r;
    o.w[0] = w0; o.w[1] = w1; o.w[2] = w2;
    o.s_lam = o.s_a = o.s_k = 1.f;
    o.s_w[0] = o.s_w[1] = o.s_w[2] = 1.f;
    return;
  }
  o.lam = expf(lam_r);
  o.s_lam = o.lam;
  o.a = expf(a_r);
  o.s_a = o.a;
  // k = 20 (tanh r + 1) = 40 sig(2r); dk/dr = 20 (1 - tanh^2 r) = 80 sig (1 - sig).
  // Written through sig so that k keeps relative accuracy as tanh r -> -1.
  const float e = expf(-2.f * k_r);
  const float sig = 1.f / (1.f + e);
  const float one_m_sig = (k_r >= 0.f) ? e * sig : 1.f - sig;
  o.k = 40.f * sig;
  o.s_k = 80.f * sig * one_m_sig;
  const float wr[3] = {w0, w1, w2};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float t = tanhf(wr[c]);
    o.w[c] = t;
    o.s_w[c] = (1.f - t) * (1.f + t);
  }
}

// ---------------------------------------------------------------------------
// Frames: x and z axes of the lobe (y = z x x never formed; G does not use it)
// ---------------------------------------------------------------------------

struct QuatFrame {
  float q[4];       // normalised quaternion (w, x, y, z)
  float inv_norm;   // 1/|q_raw|
  float x[3], z[3];
};

__device__ __forceinline__ void quat_frame(float qw, float qx, float qy, float qz, QuatFrame& f) {
  const float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
  const float inv = 1.f / sqrtf(n2);
  f.inv_norm = inv;
  const float w = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
  f.q[0] = w; f.q[1] = x; f.q[2] = y; f.q[3] = z;
  // first and third columns of the rotation matrix of the unit quaternion
  f.x[0] = 1.f - 2.f * (y * y + z * z);
  f.x[1] = 2.f * (x * y + w * z);
  f.x[2] = 2.f * (x * z - w * y);
  f.z[0] = 2.f * (x * z + w * y);
  f.z[1] = 2.f * (y * z - w * x);
  f.z[2] = 1.f - 2.f * (x * x + y * y);
}

// dLoss/dq_raw from dLoss/dx and dLoss/dz (through the unit-quaternion
// rotation columns and the normalisation q -> q/|q|).
__device__ __forceinline__ void quat_frame_grad(const QuatFrame& f, const float L[3], const float M[3],
                                                float g[4]) {
  const float w = f.q[0], x = f.q[1], y = f.q[2], z = f.q[3];
  float gw = 2.f * (L[1] * z - L[2] * y + M[0] * y - M[1] * x);
  float gx = 2.f * (L[1] * y + L[2] * z + M[0] * z - M[1] * w - 2.f * M[2] * x);
  float gy = 2.f * (-2.f * L[0] * y + L[1] * x - L[2] * w + M[0] * w + M[1] * z - 2.f * M[2] * y);
  float gz = 2.f * (-2.f * L[0] * z + L[1] * w + L[2] * x + M[0] * x + M[1] * y);
  const float dot = gw * w + gx * x + gy * y + gz * z;
  g[0] = (gw - dot * w) * f.inv_norm;
  g[1] = (gx - dot * x) * f.inv_norm;
  g[2] = (gy - dot * y) * f.inv_norm;
  g[3] = (gz - dot * z) * f.inv_norm;
}

// Supp. C frame from three cosines. RAW mode: c = tanh(r), s = sech(r) >= 0,
// with dc/dr = s^2 and ds/dr = -c s (finite everywhere, including where tanh
// saturates). IDENTITY mode: c = r, s = sqrt(1 - c^2), ds/dc = -c/s.
struct CosFrame {
  float c[3], s[3];     // cos / sin of theta, phi, psi
  float dc[3], ds[3];   // d c / d stored, d s / d stored
  float x[3], z[3];
};

__device__ __forceinline__ void cos_angle(float r, bool identity, float& c, float& s, float& dc, float& ds) {
  if (identity) {
    c = r;
    s = sqrtf(fmaxf(0.f, (1.f - r) * (1.f + r)));
    dc = 1.f;
    ds = -c / s;
    return;
  }
  const float ar = fabsf(r);
  const float em = expf(-ar);                // e^{-|r|}
  const float inv = 1.f / (1.f + em * em);
  const float t = -expm1f(-2.f * ar) * inv;  // tanh|r|
  c = copysignf(t, r);
  s = 2.f * em * inv;                        // sech r
  dc = s * s;
  ds = -c * s;
}

__device__ __forceinline__ void cos_frame(float rt, float rp, float rs, bool identity, CosFrame& f) {
  cos_angle(rt, identity, f.c[0], f.s[0], f.dc[0], f.ds[0]);
  cos_angle(rp, identity, f.c[1], f.s[1], f.dc[1], f.ds[1]);
  cos_angle(rs, identity, f.c[2], f.s[2], f.dc[2], f.ds[2]);
  const float ct = f.c[0], st = f.s[0], cp = f.c[1], sp = f.s[1], cs = f.c[2], ss = f.s[2];
  f.z[0] = ct * sp; f.z[1] = st * sp; f.z[2] = cp;
  f.x[0] = ct * cp * cs - st * ss;
  f.x[1] = st * cp * cs + ct * ss;
  f.x[2] = -sp * cs;
}

__device__ __forceinline__ void cos_frame_grad(const CosFrame& f, const float gx[3], const float gz[3],
                                               float g[3]) {
  const float ct = f.c[0], st = f.s[0], cp = f.c[1], sp = f.s[1], cs = f.c[2], ss = f.s[2];
  const float g_ct = gx[0] * cp * cs + gx[1] * ss + gz[0] * sp;
  const float g_st = -gx[0] * ss + gx[1] * cp * cs + gz[1] * sp;
  const float g_cp = gx[0] * ct * cs + gx[1] * st * cs + gz[2];
  const float g_sp = -gx[2] * cs + gz[0] * ct + gz[1] * st;
  const float g_cs = gx[0] * ct * cp + gx[1] * st * cp - gx[2] * sp;
  const float g_ss = -gx[0] * st + gx[1] * ct;
  g[0] = g_ct * f.dc[0] + g_st * f.ds[0];
  g[1] = g_cp * f.dc[1] + g_sp * f.ds[1];
  g[2] = g_cs * f.dc[2] + g_ss * f.ds[2];
}

// ---------------------------------------------------------------------------
// The lobe and its partial derivatives
// ---------------------------------------------------------------------------

struct LobePartials {
  float G_u, G_v, G_lam, G_a, G_k;  // dG/du, dG/dv, dG/dlam, dG/da, dG/dk
};

template <bool GRAD>
__device__ __forceinline__ float lobe(const float d[3], const float x[3], const float z[3], float lam,
                                      float a, float k, bool normalised, LobePartials* pd) {
  const float u = d[0] * z[0] + d[1] * z[1] + d[2] * z[2];
  const float v = d[0] * x[0] + d[1] * x[1] + d[2] * x[2];
  const float cx = d[1] * z[2] - d[2] * z[1];
  const float cy = d[2] * z[0] - d[0] * z[2];
  const float cz = d[0] * z[1] - d[1] * z[0];
  const float s2 = cx * cx + cy * cy + cz * cz;  // 1 - u^2
  const bool pole = !(s2 > 0.f);
  const bool anti = pole && (u < 0.f);
  const float inv_s2 = pole ? 0.f : 1.f / s2;
  const float omu = (u >= 0.f) ? s2 / (1.f + u) : 1.f - u;  // 1 - u
  const float ln_k = anti ? 0.f : log1pf(-0.5f * omu);      // ln kappa
  const float tau = a * v * v * inv_s2;
  const float ln_e = tau * ln_k;                            // ln E
  const float em1 = expm1f(ln_e + ln_k);                    // E kappa - 1
  const float pe = expf(2.f * lam * em1 + ln_e);            // p E
  float sh, ch;
  sincosf(0.5f * k * v, &sh, &ch);
  const float h = ch * ch;
  float cinv = 1.f, dlnc_dlam = 0.f, dlnc_da = 0.f;
  if (normalised) {
    const float em = expm1f(-2.f * lam);  // e^{-2 lam} - 1 (negative)
    const float sq = sqrtf(1.f + a);
    cinv = lam * sq * kInvTwoPi / (-em);
    if (GRAD) {
      // d ln C^-1/d lam = 1/lam - 2 e^{-2 lam}/(1 - e^{-2 lam}); d ln C^-1/d a = 1/(2 (1+a))
      dlnc_dlam = 1.f / lam + 2.f * (1.f + em) / em;
      dlnc_da = 0.5f / (1.f + a);
    }
  }
  const float cpe = cinv * pe;
  const float G = anti ? 0.f : cpe * h;
  if (GRAD) {
    if (anti) {
      pd->G_u = pd->G_v = pd->G_lam = pd->G_a = pd->G_k = 0.f;
    } else {
      // 1/(1+u) = 1/(2 kappa); for u < 0, 1 + u = s2/(1 - u) without cancellation
      const float inv_opu = (u >= 0.f) ? 1.f / (1.f + u) : (1.f - u) * inv_s2;
      const float ek = em1 + 1.f;                       // E kappa
      const float two_lam_ek = 2.f * lam * ek;
      const float dtau_du = 2.f * u * tau * inv_s2;
      const float dtau_dv = 2.f * a * v * inv_s2;
      const float dlne_du = ln_k * dtau_du + tau * inv_opu;
      const float dlne_dv = ln_k * dtau_dv;
      const float sin_kv = 2.f * sh * ch;
      pd->G_u = G * (two_lam_ek * (dlne_du + inv_opu) + dlne_du);
      pd->G_v = G * (two_lam_ek + 1.f) * dlne_dv - cpe * (0.5f * k) * sin_kv;
      pd->G_k = -cpe * (0.5f * v) * sin_kv;
      pd->G_lam = G * (2.f * em1 + dlnc_dlam);
      pd->G_a = G * ((two_lam_ek + 1.f) * ln_k * v * v * inv_s2 + dlnc_da);
    }
  }
  return G;
}

// ---------------------------------------------------------------------------
// View direction d = (mu - cam)/|mu - cam|
// ---------------------------------------------------------------------------

__device__ __forceinline__ float view_dir(const float* means, int64_t i, float cx, float cy, float cz,
                                          float d[3]) {
  const float rx = __ldg(means + 3 * i + 0) - cx;
  const float ry = __ldg(means + 3 * i + 1) - cy;
  const float rz = __ldg(means + 3 * i + 2) - cz;
  const float dist = sqrtf(rx * rx + ry * ry + rz * rz);
  const float inv = 1.f / dist;
  d[0] = rx * inv; d[1] = ry * inv; d[2] = rz * inv;
  return inv;
}

// dLoss/dmu = (I - d d^T) dLoss/dd / |mu - cam|
__device__ __forceinline__ void dir_grad(const float d[3], const float gd[3], float inv_dist, float gm[3]) {
  const float dot = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
  gm[0] = (gd[0] - dot * d[0]) * inv_dist;
  gm[1] = (gd[1] - dot * d[1]) * inv_dist;
  gm[2] = (gd[2] - dot * d[2]) * inv_dist;
}

}  // namespace nasg
