// Bond-dimension extrapolation of observables: a least-squares fit linear in
// 1/chi per observable, the chi -> infinity estimate being the intercept (the
// linear extrapolation in 1/chi of the n = 20 results, Fig. F2c).
#include <cmath>
#include <vector>

#include "tnbp.h"

extern "C" tn_status tn_chi_extrapolate(const double* chi, const double* values, int32_t n_chi,
                                        int32_t n_obs, double* intercept, double* slope,
                                        double* rms) {
  if (!chi || !values || !intercept || n_chi < 2 || n_obs < 1) return TN_EINVAL;
  std::vector<double> x(n_chi);
  double xm = 0.0;
  for (int32_t i = 0; i < n_chi; ++i) {
    if (!(chi[i] > 0.0) || !std::isfinite(chi[i])) return TN_EINVAL;
    x[i] = 1.0 / chi[i];
    xm += x[i];
  }
  xm /= n_chi;
  double sxx = 0.0;
  for (int32_t i = 0; i < n_chi; ++i) sxx += (x[i] - xm) * (x[i] - xm);
  if (!(sxx > 0.0)) return TN_EINVAL;  // every chi the same: no slope to fit
  for (int64_t i = 0; i < (int64_t)n_chi * n_obs; ++i)
    if (!std::isfinite(values[i])) return TN_EINVAL;
  for (int32_t k = 0; k < n_obs; ++k) {
    double ym = 0.0;
    for (int32_t i = 0; i < n_chi; ++i) ym += values[(int64_t)i * n_obs + k];
    ym /= n_chi;
    double sxy = 0.0;
    for (int32_t i = 0; i < n_chi; ++i) sxy += (x[i] - xm) * (values[(int64_t)i * n_obs + k] - ym);
    const double b = sxy / sxx, a = ym - b * xm;
    intercept[k] = a;
    if (slope) slope[k] = b;
    if (rms) {
      double r2 = 0.0;
      for (int32_t i = 0; i < n_chi; ++i) {
        const double d = values[(int64_t)i * n_obs + k] - (a + b * x[i]);
        r2 += d * d;
      }
      rms[k] = std::sqrt(r2 / n_chi);
    }
  }
  return TN_OK;
}
