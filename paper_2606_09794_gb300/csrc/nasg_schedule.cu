// Learning-rate rules of the method, host side (nasg_lr_heuristic,
// nasg_cosine_lr_factor): small per-scene / per-iteration scalars that feed the
// Adam learning rates of the fused step and fitting kernels.
//
// Sec. 4.2 heuristic: d_knn is the mean over cameras of the mean distance from
// a camera centre to its k nearest other camera centres; the appearance
// (feature) rate scales as (d_ref / d_knn)^beta and the opacity rate as
// (d_knn / d_ref)^gamma. Supp. C scheduling: a cosine factor
// (1 + cos(pi s / S)) / 2 over the scheduled part of training.
#include <algorithm>
#include <cmath>
#include <vector>

#include "nasgabor.h"

extern "C" nasg_status nasg_lr_heuristic(const float* centres, int32_t n_cams, int32_t k, double d_ref,
                                         double eta_f_base, double eta_sigma_base, double beta, double gamma,
                                         double* eta_f, double* eta_sigma, double* d_knn) {
  if (!centres || !eta_f || !eta_sigma) return NASG_ERR_NULL;
  if (n_cams < 2 || k < 1 || !(d_ref > 0.0) || !std::isfinite(d_ref)) return NASG_ERR_RANGE;
  const int kk = std::min<int>(k, n_cams - 1);
  std::vector<double> dist(size_t(n_cams) - 1);
  double total = 0.0;
  for (int i = 0; i < n_cams; ++i) {
    int m = 0;
    for (int j = 0; j < n_cams; ++j) {
      if (j == i) continue;
      double s = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double d = double(centres[3 * i + c]) - double(centres[3 * j + c]);
        s += d * d;
      }
      dist[m++] = std::sqrt(s);
    }
    std::partial_sort(dist.begin(), dist.begin() + kk, dist.end());
    double mean = 0.0;
    for (int j = 0; j < kk; ++j) mean += dist[j];
    total += mean / kk;
  }
  const double d = total / n_cams;
  if (!(d > 0.0) || !std::isfinite(d)) return NASG_ERR_RANGE;  // coincident cameras
  *eta_f = eta_f_base * std::pow(d_ref / d, beta);
  *eta_sigma = eta_sigma_base * std::pow(d / d_ref, gamma);
  if (d_knn) *d_knn = d;
  return NASG_OK;
}

extern "C" double nasg_cosine_lr_factor(int64_t t, int64_t t_start, int64_t t_max) {
  if (t < t_start) return 1.0;
  const int64_t span = t_max - t_start;
  const int64_t s = t - t_start;
  if (span <= 0 || s >= span) return 0.0;
  return 0.5 * (1.0 + std::cos(M_PI * double(s) / double(span)));
}
