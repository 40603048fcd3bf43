// Value types for the lobe math: a scalar float, or P2 = two lobes' values in
// one float2 whose add/mul/fma map to sm_100's packed FP32 instructions
// (one issue slot for two operations). Comparisons on P2 give B2 masks and
// selects are per component. The transcendental building blocks use the
// hardware approximations (ex2/lg2/rcp/rsqrt .approx.ftz) through inline PTX,
// component by component.
#pragma once

#include <cuda_runtime.h>

namespace nasg {

// ---- hardware approximations (MUFU) ---------------------------------------
__device__ __forceinline__ float ex2a(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2a(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcpa(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqa(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---- packed pair -------------------------------------------------------------
struct P2 {
  float2 v;
};
struct B2 {
  bool x, y;
};

__device__ __forceinline__ P2 p2(float a) { P2 r; r.v = make_float2(a, a); return r; }
__device__ __forceinline__ P2 p2(float a, float b) { P2 r; r.v = make_float2(a, b); return r; }

__device__ __forceinline__ P2 operator+(P2 a, P2 b) { P2 r; r.v = __fadd2_rn(a.v, b.v); return r; }
__device__ __forceinline__ P2 operator*(P2 a, P2 b) { P2 r; r.v = __fmul2_rn(a.v, b.v); return r; }
__device__ __forceinline__ P2 operator-(P2 a, P2 b) {
  P2 r;
  r.v = __ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v);
  return r;
}
__device__ __forceinline__ P2 operator-(P2 a) { return p2(-a.v.x, -a.v.y); }
__device__ __forceinline__ P2 operator+(P2 a, float b) { return a + p2(b); }
__device__ __forceinline__ P2 operator+(float a, P2 b) { return p2(a) + b; }
__device__ __forceinline__ P2 operator-(P2 a, float b) { return a - p2(b); }
__device__ __forceinline__ P2 operator-(float a, P2 b) { return p2(a) - b; }
__device__ __forceinline__ P2 operator*(P2 a, float b) { return a * p2(b); }
__device__ __forceinline__ P2 operator*(float a, P2 b) { return p2(a) * b; }

__device__ __forceinline__ P2 vfma(P2 a, P2 b, P2 c) { P2 r; r.v = __ffma2_rn(a.v, b.v, c.v); return r; }
__device__ __forceinline__ P2 vfma(P2 a, float b, P2 c) { return vfma(a, p2(b), c); }
__device__ __forceinline__ P2 vfma(P2 a, P2 b, float c) { return vfma(a, b, p2(c)); }
__device__ __forceinline__ P2 vfma(P2 a, float b, float c) { return vfma(a, p2(b), p2(c)); }
__device__ __forceinline__ P2 vfma(float a, P2 b, P2 c) { return vfma(p2(a), b, c); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }

// ---- per-component operations -------------------------------------------------
#define NASG_MAP1(NAME, EXPR)                                                      \
  __device__ __forceinline__ float NAME(float a) { return EXPR(a); }              \
  __device__ __forceinline__ P2 NAME(P2 a) { return p2(EXPR(a.v.x), EXPR(a.v.y)); }
NASG_MAP1(vex2, ex2a)
NASG_MAP1(vlg2, lg2a)
NASG_MAP1(vrcp, rcpa)
NASG_MAP1(vrsqrt, rsqa)
NASG_MAP1(vabs, fabsf)
NASG_MAP1(vrint, rintf)
#undef NASG_MAP1

__device__ __forceinline__ float vcopysign(float a, float b) { return copysignf(a, b); }
__device__ __forceinline__ P2 vcopysign(P2 a, P2 b) {
  return p2(copysignf(a.v.x, b.v.x), copysignf(a.v.y, b.v.y));
}
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ P2 vmin(P2 a, float b) { return p2(fminf(a.v.x, b), fminf(a.v.y, b)); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ P2 vmax(P2 a, float b) { return p2(fmaxf(a.v.x, b), fmaxf(a.v.y, b)); }

__device__ __forceinline__ bool vge(float a, float b) { return a >= b; }
__device__ __forceinline__ B2 vge(P2 a, float b) { return {a.v.x >= b, a.v.y >= b}; }
__device__ __forceinline__ bool vgt(float a, float b) { return a > b; }
__device__ __forceinline__ B2 vgt(P2 a, float b) { return {a.v.x > b, a.v.y > b}; }
__device__ __forceinline__ bool vlt(float a, float b) { return a < b; }
__device__ __forceinline__ B2 vlt(P2 a, float b) { return {a.v.x < b, a.v.y < b}; }
__device__ __forceinline__ bool vand(bool a, bool b) { return a && b; }
__device__ __forceinline__ B2 vand(B2 a, B2 b) { return {a.x && b.x, a.y && b.y}; }
__device__ __forceinline__ bool vnot(bool a) { return !a; }
__device__ __forceinline__ B2 vnot(B2 a) { return {!a.x, !a.y}; }

__device__ __forceinline__ float vsel(bool m, float a, float b) { return m ? a : b; }
__device__ __forceinline__ P2 vsel(B2 m, P2 a, P2 b) { return p2(m.x ? a.v.x : b.v.x, m.y ? a.v.y : b.v.y); }
__device__ __forceinline__ P2 vsel(B2 m, float a, P2 b) { return p2(m.x ? a : b.v.x, m.y ? a : b.v.y); }
__device__ __forceinline__ P2 vsel(B2 m, P2 a, float b) { return p2(m.x ? a.v.x : b, m.y ? a.v.y : b); }

// integer quadrant of a rounded float (for sincos)
__device__ __forceinline__ int vquad(float n) { return static_cast<int>(n) & 3; }

template <class V>
__device__ __forceinline__ V vconst(float c);
template <>
__device__ __forceinline__ float vconst<float>(float c) { return c; }
template <>
__device__ __forceinline__ P2 vconst<P2>(float c) { return p2(c); }

template <class V>
struct VecTraits;
template <>
struct VecTraits<float> {
  using Mask = bool;
};
template <>
struct VecTraits<P2> {
  using Mask = B2;
};

}  // namespace nasg
