// Real spherical harmonics, degree 0..3 (Sec. 3.2 of arXiv 2606.09794: the
// comparison appearance model f(d; c) = sum_lm c_lm Y_l^m(d)), forward and
// backward, with their C ABI entry points (sh_eval_fwd / sh_eval_bwd).
//
// Basis: orthonormal real SH with the Condon-Shortley phase,
//   Y_lm = sqrt(2) K_lm P_l^m(cos t) cos(m p)  (m > 0), K_l0 P_l(cos t) (m = 0),
//   sqrt(2) K_l|m| P_l^|m|(cos t) sin(|m| p)    (m < 0),
// K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), index j = l^2 + l + m. Written out
// as polynomials in the unit direction (x, y, z); each constant is stated with
// its closed form. The gradient wrt d uses the polynomials' Cartesian
// gradients, projected onto the sphere's tangent plane by the direction chain
// (I - d d^T)/|mu - cam|, which removes any radial part.
//
// Mapping: one thread per primitive; coefficient planes [j][c][N] are read
// with unit stride across the warp.
#include "nasg_device.cuh"
#include "nasg_host.h"

namespace nasg {

// closed forms of the normalisation constants
constexpr float kY00 = 0.282094791773878143f;   // 1/(2 sqrt(pi))
constexpr float kY1 = 0.488602511902919921f;    // sqrt(3/(4 pi))
constexpr float kY2a = 1.092548430592079070f;   // sqrt(15/(4 pi))
constexpr float kY2b = 0.315391565252520050f;   // sqrt(5/(16 pi))
constexpr float kY2c = 0.546274215296039535f;   // sqrt(15/(16 pi))
constexpr float kY3a = -0.590043589926643510f;  // -sqrt(35/(32 pi))
constexpr float kY3b = 2.890611442640554055f;   // sqrt(105/(4 pi))
constexpr float kY3c = -0.457045799464465737f;  // -sqrt(21/(32 pi))
constexpr float kY3d = 0.373176332590115391f;   // sqrt(7/(16 pi))
constexpr float kY3e = 1.445305721320277027f;   // sqrt(105/(16 pi))

// Y_j (j < (DEG+1)^2) and, with GRAD, the Cartesian gradient of each polynomial.
template <int DEG, bool GRAD>
__device__ __forceinline__ void sh_basis(const float d[3], float* Y, float (*dY)[3]) {
  const float x = d[0], y = d[1], z = d[2];
  Y[0] = kY00;
  if (GRAD) { dY[0][0] = dY[0][1] = dY[0][2] = 0.f; }
  if (DEG >= 1) {
    Y[1] = -kY1 * y;
    Y[2] = kY1 * z;
    Y[3] = -kY1 * x;
    if (GRAD) {
      dY[1][0] = 0.f; dY[1][1] = -kY1; dY[1][2] = 0.f;
      dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = kY1;
      dY[3][0] = -kY1; dY[3][1] = 0.f; dY[3][2] = 0.f;
    }
  }
  if (DEG >= 2) {
    Y[4] = kY2a * x * y;
    Y[5] = -kY2a * y * z;
    Y[6] = kY2b * (3.f * z * z - 1.f);
    Y[7] = -kY2a * x * z;
    Y[8] = kY2c * (x * x - y * y);
    if (GRAD) {
      dY[4][0] = kY2a * y; dY[4][1] = kY2a * x; dY[4][2] = 0.f;
      dY[5][0] = 0.f; dY[5][1] = -kY2a * z; dY[5][2] = -kY2a * y;
      dY[6][0] = 0.f; dY[6][1] = 0.f; dY[6][2] = 6.f * kY2b * z;
      dY[7][0] = -kY2a * z; dY[7][1] = 0.f; dY[7][2] = -kY2a * x;
      dY[8][0] = 2.f * kY2c * x; dY[8][1] = -2.f * kY2c * y; dY[8][2] = 0.f;
    }
  }
  if (DEG >= 3) {
    const float z2 = z * z;
    Y[9] = kY3a * y * (3.f * x * x - y * y);
    Y[10] = kY3b * x * y * z;
    Y[11] = kY3c * y * (5.f * z2 - 1.f);
    Y[12] = kY3d * z * (5.f * z2 - 3.f);
    Y[13] = kY3c * x * (5.f * z2 - 1.f);
    Y[14] = kY3e * z * (x * x - y * y);
    Y[15] = kY3a * x * (x * x - 3.f * y * y);
    if (GRAD) {
      dY[9][0] = kY3a * 6.f * x * y; dY[9][1] = kY3a * 3.f * (x * x - y * y); dY[9][2] = 0.f;
      dY[10][0] = kY3b * y * z; dY[10][1] = kY3b * x * z; dY[10][2] = kY3b * x * y;
      dY[11][0] = 0.f; dY[11][1] = kY3c * (5.f * z2 - 1.f); dY[11][2] = kY3c * 10.f * y * z;
      dY[12][0] = 0.f; dY[12][1] = 0.f; dY[12][2] = kY3d * (15.f * z2 - 3.f);
      dY[13][0] = kY3c * (5.f * z2 - 1.f); dY[13][1] = 0.f; dY[13][2] = kY3c * 10.f * x * z;
      dY[14][0] = kY3e * 2.f * x * z; dY[14][1] = -kY3e * 2.f * y * z; dY[14][2] = kY3e * (x * x - y * y);
      dY[15][0] = kY3a * 3.f * (x * x - y * y); dY[15][1] = -kY3a * 6.f * x * y; dY[15][2] = 0.f;
    }
  }
}

struct ShArgs {
  int64_t n;
  const float* coeffs;
  const float* means;
  float cam[3];
  const float* g_rgb;
  float* rgb;
  float* g_coeffs;
  float* g_means;
};

template <int DEG>
__global__ void __launch_bounds__(256) sh_fwd_kernel(const ShArgs a) {
  constexpr int NB = (DEG + 1) * (DEG + 1);
  const int64_t n = a.n;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    float d[3];
    view_dir(a.means, i, a.cam[0], a.cam[1], a.cam[2], d);
    float Y[NB];
    sh_basis<DEG, false>(d, Y, nullptr);
    float rgb[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < NB; ++j) {
#pragma unroll
      for (int c = 0; c < 3; ++c) rgb[c] = fmaf(__ldg(a.coeffs + (int64_t(j) * 3 + c) * n + i), Y[j], rgb[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) a.rgb[3 * i + c] = rgb[c];
  }
}

template <int DEG>
// 64 registers (4 blocks of 256 threads per SM): with all 48 coefficient loads of
// a thread issued before its first use, occupancy and loads in flight together
// keep HBM busy (at 255 registers, one block per SM, it ran at 40 % of the copy
// bandwidth; interleaved with the stores, at 65 %).
__global__ void __launch_bounds__(256, 4) sh_bwd_kernel(const ShArgs a) {
  constexpr int NB = (DEG + 1) * (DEG + 1);
  const int64_t n = a.n;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    float d[3];
    const float inv_dist = view_dir(a.means, i, a.cam[0], a.cam[1], a.cam[2], d);
    float Y[NB];
    float dY[NB][3];
    sh_basis<DEG, true>(d, Y, dY);
    float g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c] = __ldg(a.g_rgb + 3 * i + c);
    // dLoss/dd first (coefficient loads only), then the gradient stores: the
    // compiler may not move a load of coeffs past a store to g_coeffs (they could
    // alias), so interleaving the two would leave one load in flight per thread.
    float gd[3] = {0.f, 0.f, 0.f};
    if (a.g_means) {
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        float gy = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) gy = fmaf(g[c], __ldg(a.coeffs + (int64_t(j) * 3 + c) * n + i), gy);
#pragma unroll
        for (int k = 0; k < 3; ++k) gd[k] = fmaf(gy, dY[j][k], gd[k]);
      }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c) a.g_coeffs[(int64_t(j) * 3 + c) * n + i] = g[c] * Y[j];
    if (a.g_means) {
      float gm[3];
      dir_grad(d, gd, inv_dist, gm);
#pragma unroll
      for (int c = 0; c < 3; ++c) a.g_means[3 * i + c] = gm[c];
    }
  }
}

template <bool BWD>
static nasg_status launch_sh(int degree, const ShArgs& a, cudaStream_t s) {
  constexpr int kBlock = 256;
  const unsigned grid = grid_for(a.n, kBlock);
  switch (degree) {
#define NASG_SH_CASE(D)                                                   \
  case D:                                                                 \
    if (BWD) sh_bwd_kernel<D><<<grid, kBlock, 0, s>>>(a);                 \
    else sh_fwd_kernel<D><<<grid, kBlock, 0, s>>>(a);                     \
    break;
    NASG_SH_CASE(0)
    NASG_SH_CASE(1)
    NASG_SH_CASE(2)
    NASG_SH_CASE(3)
#undef NASG_SH_CASE
    default:
      return NASG_ERR_RANGE;
  }
  return check_launch();
}

}  // namespace nasg

using namespace nasg;

extern "C" nasg_status sh_eval_fwd(int32_t degree, int64_t n, const float* coeffs, const float* means,
                                   const float* cam, float* rgb, void* stream) {
  if (degree < 0 || degree > 3 || n < 0) return NASG_ERR_RANGE;
  if (n == 0) return NASG_OK;
  if (!coeffs || !means || !cam || !rgb) return NASG_ERR_NULL;
  if (!aligned(coeffs, 4) || !aligned(means, 4) || !aligned(rgb, 4)) return NASG_ERR_ALIGN;
  if (n == 0) return NASG_OK;
  ShArgs a{};
  a.n = n;
  a.coeffs = coeffs;
  a.means = means;
  a.cam[0] = cam[0]; a.cam[1] = cam[1]; a.cam[2] = cam[2];
  a.rgb = rgb;
  return launch_sh<false>(degree, a, as_stream(stream));
}

extern "C" nasg_status sh_eval_bwd(int32_t degree, int64_t n, const float* coeffs, const float* means,
                                   const float* cam, const float* g_rgb, float* g_coeffs, float* g_means,
                                   void* stream) {
  if (degree < 0 || degree > 3 || n < 0) return NASG_ERR_RANGE;
  if (n == 0) return NASG_OK;
  if (!coeffs || !means || !cam || !g_rgb || !g_coeffs) return NASG_ERR_NULL;
  if (!aligned(coeffs, 4) || !aligned(means, 4) || !aligned(g_rgb, 4) || !aligned(g_coeffs, 4) ||
      (g_means && !aligned(g_means, 4)))
    return NASG_ERR_ALIGN;
  if (n == 0) return NASG_OK;
  ShArgs a{};
  a.n = n;
  a.coeffs = coeffs;
  a.means = means;
  a.cam[0] = cam[0]; a.cam[1] = cam[1]; a.cam[2] = cam[2];
  a.g_rgb = g_rgb;
  a.g_coeffs = g_coeffs;
  a.g_means = g_means;
  return launch_sh<true>(degree, a, as_stream(stream));
}
