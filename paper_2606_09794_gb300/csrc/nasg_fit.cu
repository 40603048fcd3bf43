// One step of fitting a student NASGabor mixture to a teacher field
// (nasgabor_fit_step): for D view directions shared by all primitives, the
// per-primitive loss is the mean over (direction, channel) of the squared
// difference between the student's and the teacher's colour (eq:app_model,
// both with the Sec. 5.1 / Supp. E-F lobe); its gradient, summed over the
// directions (Supp. F derivatives), drives one Adam step of every primitive's
// student parameters (FP32 master, BF16 copy) in the same pass. The summed
// squared error of the step is reduced per block and then deterministically
// to the mean (the loss value).
//
// Mapping: a slice of S lanes per primitive, each lane two student lobes
// (packed FP32x2). Activations, frames and the normalisation factors (which do
// not depend on the direction) are formed once per step; the direction loop
// carries only what each direction needs (frame axes, activated values,
// normalisation factors). The gradient is linear in the per-direction partials,
// so the lane accumulates dLoss/dlam, /da, /dk, /dw and dLoss/dx, dLoss/dz over
// the directions; after the loop it reloads its FP32 master values (which the
// Adam update reads anyway), forms the activation slopes and the quaternion
// frame from them again, and applies the chain once, so that none of those
// quantities stays live across the loop.
// The teacher's lobe pairs (Lt/2 of them) are spread over the slice: for a
// group of G = S/(Lt/2) directions, lane g evaluates teacher pair g % (Lt/2) at
// direction g / (Lt/2), and the teacher colours are exchanged by shuffles.
#include <cmath>

#include "nasg_kernels.cuh"

namespace nasg {

struct FitArgs {
  float* master;  // student [P][N*Ls]
  float* m;
  float* v;
  uint16_t* pbf;  // nullable
  float* c0;      // student [3][N]
  float* c0m;
  float* c0v;
  uint16_t* c0bf;  // nullable
  const float* teacher;  // [P][N*Lt] raw f32
  const float* tc0;      // [3][N]
  const float* dirs;     // [D][3]
  int64_t n;
  int32_t ls, lt, n_dirs, slice_log2;
  float b1, b2, omb1, omb2, step_size, inv_sqrt_bc2, eps;
  int32_t quantize, identity, normalised, exact;
  float* partials;  // [gridDim.x] summed squared errors
};

constexpr int kFitBlock = 256;
constexpr int kFitMaxGrid = 4096;

__device__ __forceinline__ float fit_bf16_rne(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint16_t fit_bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ void fit_adam(const FitArgs& s, float g, float& th, float& m, float& v) {
  m = fmaf(s.b1, m, s.omb1 * g);
  v = fmaf(s.b2, v, s.omb2 * (g * g));
  float sq;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sq) : "f"(v));
  const float den = fmaf(sq, s.inv_sqrt_bc2, s.eps);
  th = fmaf(-s.step_size, m * rcpa(den), th);
}

// The per-step quantities of a lobe pair that its evaluation at each direction needs.
struct FitLobes {
  P2 x[3], z[3];
  P2 lam, a, k, w[3];
  LobeNorm<P2> nc;
};

template <bool GRAD, bool EXACT>
__device__ __forceinline__ void fit_lobes(const P2* raw, bool identity, bool normalised, FitLobes& f) {
  Act<P2> act;
  activate(raw + 4, identity, act);
  QuatFrame<P2> qf;
  quat_frame(raw, qf);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    f.x[c] = qf.x[c];
    f.z[c] = qf.z[c];
    f.w[c] = act.w[c];
  }
  f.lam = act.lam;
  f.a = act.a;
  f.k = act.k;
  lobe_norm<GRAD, kFamNasGabor>(act.lam, act.a, act.k, p2(0.f), normalised, EXACT, !identity, f.nc);
}

// A float2 load the compiler may not merge with an earlier load of the same address
// (so that values reloaded after the direction loop are not kept live across it).
__device__ __forceinline__ float2 ld_f2_fresh(const float* p) {
  float2 v;
  asm volatile("ld.global.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}

// Loads the pair (2g, 2g+1) of lobes of primitive i from [P][N*L] raw planes.
__device__ __forceinline__ void load_pair(const float* planes, int64_t n, int L, int64_t i, int l0, bool quant,
                                          P2* out) {
  const int64_t NL = n * L;
  const int64_t off = i * L + l0;
#pragma unroll
  for (int p = 0; p < 10; ++p) {
    const float2 w = *reinterpret_cast<const float2*>(planes + p * NL + off);
    out[p] = quant ? p2(fit_bf16_rne(w.x), fit_bf16_rne(w.y)) : p2(w.x, w.y);
  }
}

// EXACT: exact normalisation, a compile-time choice so that the approximate
// (default) mode carries none of its code. LSC, LTC: the student and teacher lobe
// counts when fixed at compile time (0: read from the arguments), which makes the
// slice width, the teacher grouping and their loops constants.
template <bool EXACT, int LSC, int LTC>
__global__ void __launch_bounds__(kFitBlock, 2) fit_kernel(const FitArgs s) {
  __shared__ float block_sum[kFitBlock / 32];
  const int ls = LSC ? LSC : s.ls, lt = LTC ? LTC : s.lt;
  const int slog = LSC ? log2_of(slice_of_lobes(LSC)) : s.slice_log2;
  const int S = 1 << slog;
  const int g = threadIdx.x & (S - 1);
  const int l0 = 2 * g;
  const int tpairs = lt >> 1;    // teacher pairs
  const int G = S / tpairs;      // directions per teacher group
  const int tp = g % tpairs, tk = g / tpairs;
  const int lane = threadIdx.x & 31;
  const int slice0 = lane & ~(S - 1);
  const int64_t total = s.n << slog;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const float inv3d = 2.f / (3.f * float(s.n_dirs));
  float sq_sum = 0.f;
  for (int64_t t0 = int64_t(blockIdx.x) * blockDim.x; t0 < total; t0 += stride) {  // block-uniform
    const int64_t t = t0 + threadIdx.x;
    const bool ok = t < total;
    const int64_t i = ok ? (t >> slog) : 0;
    const bool mine = ok && l0 < ls;
    // ---- per-step quantities of the lane's student and teacher pairs ----
    FitLobes stu, tea;
    {
      P2 raw[10];
      if (mine) load_pair(s.master, s.n, ls, i, l0, s.quantize != 0, raw);
      else {
#pragma unroll
        for (int p = 0; p < 10; ++p) raw[p] = p2(p == 0 ? 1.f : 0.f);
      }
      fit_lobes<true, EXACT>(raw, s.identity != 0, s.normalised != 0, stu);
      if (!mine) {  // a lane past the last lobe pair adds nothing to the colour
#pragma unroll
        for (int c = 0; c < 3; ++c) stu.w[c] = p2(0.f);
      }
      if (ok) load_pair(s.teacher, s.n, lt, i, 2 * tp, false, raw);
      else {
#pragma unroll
        for (int p = 0; p < 10; ++p) raw[p] = p2(p == 0 ? 1.f : 0.f);
      }
      fit_lobes<false, EXACT>(raw, s.identity != 0, s.normalised != 0, tea);
    }
    float dc0[3];  // student minus teacher diffuse colour
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float cv = ok ? s.c0[c * s.n + i] : 0.f;
      dc0[c] = (s.quantize ? fit_bf16_rne(cv) : cv) - (ok ? s.tc0[c * s.n + i] : 0.f);
    }
    const P2 zero = p2(0.f);
    P2 acc_lam = zero, acc_a = zero, acc_k = zero;
    P2 acc_w[3] = {zero, zero, zero}, acc_gx[3] = {zero, zero, zero}, acc_gz[3] = {zero, zero, zero};
    float acc_c0[3] = {0.f, 0.f, 0.f};
    for (int base = 0; base < s.n_dirs; base += G) {  // uniform
      // teacher colour of direction base + tk from this lane's teacher pair
      float tcol[3] = {0.f, 0.f, 0.f};
      {
        const int j = min(base + tk, s.n_dirs - 1);
        const P2 d[3] = {p2(__ldg(s.dirs + 3 * j)), p2(__ldg(s.dirs + 3 * j + 1)), p2(__ldg(s.dirs + 3 * j + 2))};
        LobePartials<P2> pd;
        const P2 Gt = lobe_at<false, kFamNasGabor>(d, tea.x, tea.z, tea.lam, tea.a, tea.k, zero, tea.nc, EXACT,
                                                   s.identity == 0, &pd);
#pragma unroll
        for (int c = 0; c < 3; ++c) tcol[c] = fmaf(tea.w[c].v.y, Gt.v.y, tea.w[c].v.x * Gt.v.x);
        for (int o = 1; o < tpairs; o <<= 1) {
#pragma unroll
          for (int c = 0; c < 3; ++c) tcol[c] += __shfl_xor_sync(0xffffffffu, tcol[c], o);
        }
        // the teacher colour less the student-minus-teacher diffuse colour (this lane's
        // primitive is the slice's): the residual below is then one subtraction
#pragma unroll
        for (int c = 0; c < 3; ++c) tcol[c] -= dc0[c];
      }
      for (int kk = 0; kk < G && base + kk < s.n_dirs; ++kk) {  // uniform
        const int j = base + kk;
        float tc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) tc[c] = __shfl_sync(0xffffffffu, tcol[c], slice0 + kk * tpairs);
        const float dx = __ldg(s.dirs + 3 * j), dy = __ldg(s.dirs + 3 * j + 1), dz = __ldg(s.dirs + 3 * j + 2);
        const P2 d[3] = {p2(dx), p2(dy), p2(dz)};
        LobePartials<P2> pd;
        const P2 Gs = lobe_at<true, kFamNasGabor, P2, true>(d, stu.x, stu.z, stu.lam, stu.a, stu.k, zero, stu.nc,
                                                            EXACT, s.identity == 0, &pd);
        float col[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) col[c] = fmaf(stu.w[c].v.y, Gs.v.y, stu.w[c].v.x * Gs.v.x);
        for (int o = S >> 1; o >= 1; o >>= 1) {
#pragma unroll
          for (int c = 0; c < 3; ++c) col[c] += __shfl_xor_sync(0xffffffffu, col[c], o);
        }
        // the residual r = student - teacher colour; the accumulators sum r-weighted terms and
        // are scaled once after the loop by d(mean over directions and channels)/dc = 2/(3 D)
        float gc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          gc[c] = col[c] - tc[c];
          acc_c0[c] += gc[c];
        }
        if (ok && g == 0) {
#pragma unroll
          for (int c = 0; c < 3; ++c) sq_sum = fmaf(gc[c], gc[c], sq_sum);
        }
        const P2 gG = vfma(p2(gc[0]), stu.w[0], vfma(p2(gc[1]), stu.w[1], p2(gc[2]) * stu.w[2]));
        const P2 gGG = gG * Gs;  // G_u, G_a, G_lam come divided by G
#pragma unroll
        for (int c = 0; c < 3; ++c) acc_w[c] = vfma(p2(gc[c]), Gs, acc_w[c]);
        acc_lam = vfma(gGG, pd.G_lam, acc_lam);
        acc_a = vfma(gGG, pd.G_a, acc_a);
        acc_k = vfma(gG, pd.G_k, acc_k);
        const P2 gv = gG * pd.G_v, gu = gGG * pd.G_u;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          acc_gx[c] = vfma(gv, d[c], acc_gx[c]);
          acc_gz[c] = vfma(gu, d[c], acc_gz[c]);
        }
      }
    }
    // ---- chain to the raw parameters and take the Adam step ----
    {
      const P2 sc = p2(inv3d);
      acc_lam = acc_lam * sc;
      acc_a = acc_a * sc;
      acc_k = acc_k * sc;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc_w[c] = acc_w[c] * sc;
        acc_gx[c] = acc_gx[c] * sc;
        acc_gz[c] = acc_gz[c] * sc;
        acc_c0[c] *= inv3d;
      }
    }
    if (mine) {
      const int64_t NL = s.n * ls;
      const int64_t off = i * ls + l0;
      // the FP32 master values, reloaded: the slopes and the frame are formed again from
      // the values the step evaluated (their BF16 rounding when quantising)
      float2 th[10];
      P2 raw[10];
#pragma unroll
      for (int p = 0; p < 10; ++p) {
        th[p] = ld_f2_fresh(s.master + p * NL + off);
        raw[p] = s.quantize ? p2(fit_bf16_rne(th[p].x), fit_bf16_rne(th[p].y)) : p2(th[p].x, th[p].y);
      }
      Act<P2> act;
      activate(raw + 4, s.identity != 0, act);
      QuatFrame<P2> qf;
      quat_frame(raw, qf);
      P2 grad[10];
      quat_frame_grad(qf, acc_gx, acc_gz, grad);
      grad[4] = acc_lam;  // the lobe partials are with respect to the stored scalars
      grad[5] = acc_a;
      grad[6] = acc_k * act.s_k;
#pragma unroll
      for (int c = 0; c < 3; ++c) grad[7 + c] = acc_w[c] * act.s_w[c];
#pragma unroll
      for (int p = 0; p < 10; ++p) {
        float2 mm = *reinterpret_cast<const float2*>(s.m + p * NL + off);
        float2 vv = *reinterpret_cast<const float2*>(s.v + p * NL + off);
        fit_adam(s, grad[p].v.x, th[p].x, mm.x, vv.x);
        fit_adam(s, grad[p].v.y, th[p].y, mm.y, vv.y);
        *reinterpret_cast<float2*>(s.master + p * NL + off) = th[p];
        *reinterpret_cast<float2*>(s.m + p * NL + off) = mm;
        *reinterpret_cast<float2*>(s.v + p * NL + off) = vv;
        if (s.pbf) {
          const uint32_t w2 = uint32_t(fit_bf16_bits(th[p].x)) | (uint32_t(fit_bf16_bits(th[p].y)) << 16);
          *reinterpret_cast<uint32_t*>(s.pbf + p * NL + off) = w2;
        }
      }
    }
    if (ok) {
      for (int c = g; c < 3; c += S) {
        const int64_t o = int64_t(c) * s.n + i;
        float th = s.c0[o], mm = s.c0m[o], vv = s.c0v[o];
        fit_adam(s, pick3(acc_c0, c), th, mm, vv);
        s.c0[o] = th;
        s.c0m[o] = mm;
        s.c0v[o] = vv;
        if (s.c0bf) s.c0bf[o] = fit_bf16_bits(th);
      }
    }
  }
  // block sum of the squared errors (fixed order: warp tree, then warps in order)
  for (int o = 16; o >= 1; o >>= 1) sq_sum += __shfl_xor_sync(0xffffffffu, sq_sum, o);
  if (lane == 0) block_sum[threadIdx.x >> 5] = sq_sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f;
    for (int w = 0; w < kFitBlock / 32; ++w) b += block_sum[w];
    s.partials[blockIdx.x] = b;
  }
}

// mean = (sum of partials, in order, in double) / count
__global__ void fit_loss_kernel(const float* partials, int n_parts, double count, float* loss) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int j = threadIdx.x; j < n_parts; j += blockDim.x) acc += double(partials[j]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o >= 1; o >>= 1) {
    if (threadIdx.x < unsigned(o)) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = float(red[0] / count);
}

}  // namespace nasg

using namespace nasg;

extern "C" size_t nasgabor_fit_workspace_bytes(void) { return size_t(kFitMaxGrid) * sizeof(float); }

extern "C" nasg_status nasgabor_fit_step(const nasg_desc* desc, const nasg_train_state* st,
                                         const float* teacher_params, const float* teacher_c0,
                                         int32_t teacher_lobes, const float* dirs, int32_t n_dirs,
                                         const nasg_adam_hparams* hp, float* loss, void* workspace,
                                         size_t workspace_bytes, void* stream) {
  nasg_status e = check_desc(desc);
  if (e != NASG_OK) return e;
  if (desc->frame_mode != NASG_FRAME_QUAT || desc->lobe_family != NASG_FAMILY_NASGABOR) return NASG_ERR_UNSUPPORTED;
  if (desc->accumulate != 0) return NASG_ERR_RANGE;
  if (!st || !hp || !loss) return NASG_ERR_NULL;
  const int ls = desc->n_lobes;
  const int sl = slice_log2(ls);
  const int S = 1 << sl;
  if (ls % 2 != 0 || teacher_lobes < 2 || teacher_lobes % 2 != 0 || teacher_lobes > NASG_MAX_LOBES)
    return NASG_ERR_UNSUPPORTED;
  const int tpairs = teacher_lobes / 2;
  if (tpairs > S || S % tpairs != 0 || (tpairs & (tpairs - 1)) != 0) return NASG_ERR_UNSUPPORTED;
  if (n_dirs < 1 || n_dirs > (1 << 20)) return NASG_ERR_RANGE;
  if (hp->step < 1 || !(hp->lr >= 0.f) || !(hp->beta1 >= 0.f && hp->beta1 < 1.f) ||
      !(hp->beta2 >= 0.f && hp->beta2 < 1.f) || !(hp->eps > 0.f))
    return NASG_ERR_RANGE;
  if (workspace_bytes < nasgabor_fit_workspace_bytes()) return NASG_ERR_RANGE;
  cudaStream_t cs = as_stream(stream);
  if (desc->n == 0) {
    if (cudaMemsetAsync(loss, 0, sizeof(float), cs) != cudaSuccess) return check_launch();
    return NASG_OK;
  }
  if (!st->master || !st->m || !st->v || !st->c0_master || !st->c0_m || !st->c0_v || !teacher_params ||
      !teacher_c0 || !dirs || !workspace)
    return NASG_ERR_NULL;
  const void* a8[] = {st->master, st->m, st->v, teacher_params};
  for (const void* p : a8)
    if (!aligned(p, 8)) return NASG_ERR_ALIGN;
  const void* a4[] = {st->c0_master, st->c0_m, st->c0_v, teacher_c0, dirs, loss, workspace};
  for (const void* p : a4)
    if (!aligned(p, 4)) return NASG_ERR_ALIGN;
  if ((st->params_bf16 && !aligned(st->params_bf16, 4)) || (st->c0_bf16 && !aligned(st->c0_bf16, 2)))
    return NASG_ERR_ALIGN;
  FitArgs a{};
  a.master = st->master;
  a.m = st->m;
  a.v = st->v;
  a.pbf = static_cast<uint16_t*>(st->params_bf16);
  a.c0 = st->c0_master;
  a.c0m = st->c0_m;
  a.c0v = st->c0_v;
  a.c0bf = static_cast<uint16_t*>(st->c0_bf16);
  a.teacher = teacher_params;
  a.tc0 = teacher_c0;
  a.dirs = dirs;
  a.n = desc->n;
  a.ls = ls;
  a.lt = teacher_lobes;
  a.n_dirs = n_dirs;
  a.slice_log2 = sl;
  const double b1 = hp->beta1, b2 = hp->beta2;
  const double bc1 = 1.0 - std::pow(b1, double(hp->step));
  const double bc2 = 1.0 - std::pow(b2, double(hp->step));
  a.b1 = float(b1);
  a.b2 = float(b2);
  a.omb1 = float(1.0 - b1);
  a.omb2 = float(1.0 - b2);
  a.step_size = float(double(hp->lr) / bc1);
  a.inv_sqrt_bc2 = float(1.0 / std::sqrt(bc2));
  a.eps = hp->eps;
  a.quantize = desc->param_dtype == NASG_DTYPE_BF16;
  a.identity = desc->act_mode == NASG_ACT_IDENTITY;
  a.normalised = desc->norm_mode != NASG_NORM_NONE;
  a.exact = desc->norm_mode == NASG_NORM_EXACT;
  a.partials = static_cast<float*>(workspace);
  // the fitting workload's shape (16 student, 4 teacher lobes) runs a fixed-count instance
  auto k = a.exact ? fit_kernel<true, 0, 0>
                   : (ls == 16 && teacher_lobes == 4 ? fit_kernel<false, 16, 4> : fit_kernel<false, 0, 0>);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFitBlock, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  int64_t grid = int64_t(sm_count()) * per_sm;
  const int64_t need = ((desc->n << sl) + kFitBlock - 1) / kFitBlock;
  if (grid > need) grid = need;
  if (grid > kFitMaxGrid) grid = kFitMaxGrid;
  k<<<unsigned(grid), kFitBlock, 0, cs>>>(a);
  fit_loss_kernel<<<1, 256, 0, cs>>>(a.partials, int(grid), double(desc->n) * double(n_dirs) * 3.0, loss);
  return check_launch();
}
