// Cosine-modulated pseudo-QMF bank design (host utility for RAVE-like models).
//
// The paper runs its method on RAVE (section 2.3), whose multiband front and
// back ends are a PQMF bank the paper does not specify.  This is the textbook
// construction (Nguyen 1994; Vaidyanathan 1993): a Kaiser-windowed sinc
// prototype p[n] whose cutoff wc makes the prototype's autocorrelation vanish
// at the lags 2*M*l, l != 0 (Lin & Vaidyanathan 1998), modulated as
//   analysis  h_b[n] = 2 p[n] cos((2b+1) pi/(2M) (n - c) + (-1)^b pi/4)
//   synthesis g_b[n] = 2 p[n] cos((2b+1) pi/(2M) (n - c) - (-1)^b pi/4)
// with c = (N-1)/2.
#include <cmath>
#include <vector>

#include "../../include/cachedconv.h"
#include "cc_runtime.h"

namespace {

// modified Bessel function of the first kind, order 0 (power series)
double bessel_i0(double x) {
  double sum = 1.0, term = 1.0;
  const double q = 0.25 * x * x;
  for (int k = 1; k < 500; ++k) {
    term *= q / ((double)k * (double)k);
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  return sum;
}

std::vector<double> prototype(int taps, double wc, double beta) {
  std::vector<double> p(taps);
  const double c = 0.5 * (taps - 1);
  const double i0b = bessel_i0(beta);
  for (int n = 0; n < taps; ++n) {
    const double m = n - c;
    const double ideal = (m == 0.0) ? wc / M_PI : std::sin(wc * m) / (M_PI * m);
    const double r = 2.0 * n / (taps - 1) - 1.0;
    const double win = bessel_i0(beta * std::sqrt(std::fmax(0.0, 1.0 - r * r))) / i0b;
    p[n] = ideal * win;
  }
  return p;
}

double lag_error(int taps, int bands, double wc, double beta) {
  const std::vector<double> p = prototype(taps, wc, beta);
  auto corr = [&](int lag) {
    double s = 0.0;
    for (int n = 0; n + lag < taps; ++n) s += p[n] * p[n + lag];
    return s;
  };
  const double r0 = corr(0);
  double worst = 0.0;
  for (int lag = 2 * bands; lag < taps; lag += 2 * bands) worst = std::fmax(worst, std::fabs(corr(lag)) / r0);
  return worst;
}

}  // namespace

extern "C" cc_status cc_pqmf_design(int32_t bands, int32_t taps, double beta, double* analysis,
                                    double* synthesis, double* cutoff) {
  if (bands < 2 || taps < 2 || beta < 0.0) return cc::fail(CC_ERR_INVALID_ARG, "bad PQMF size");
  // scan [0.3 pi/M, pi/M] around the band edge pi/(2M), then golden-section refine
  const int grid = 4000;
  const double lo = 0.3 * M_PI / bands, hi = 1.0 * M_PI / bands;
  int best = 0;
  double best_err = 1e300;
  for (int i = 0; i < grid; ++i) {
    const double w = lo + (hi - lo) * i / (grid - 1);
    const double e = lag_error(taps, bands, w, beta);
    if (e < best_err) {
      best_err = e;
      best = i;
    }
  }
  double a = lo + (hi - lo) * (best > 0 ? best - 1 : 0) / (grid - 1);
  double b = lo + (hi - lo) * (best < grid - 1 ? best + 1 : grid - 1) / (grid - 1);
  const double g = 0.5 * (std::sqrt(5.0) - 1.0);
  for (int it = 0; it < 200; ++it) {
    const double c1 = b - g * (b - a), c2 = a + g * (b - a);
    if (lag_error(taps, bands, c1, beta) < lag_error(taps, bands, c2, beta))
      b = c2;
    else
      a = c1;
  }
  const double wc = 0.5 * (a + b);
  const std::vector<double> p = prototype(taps, wc, beta);
  const double c = 0.5 * (taps - 1);
  for (int band = 0; band < bands; ++band) {
    const double phase = (band % 2 ? -1.0 : 1.0) * M_PI / 4.0;
    for (int n = 0; n < taps; ++n) {
      const double theta = (2 * band + 1) * M_PI / (2.0 * bands) * (n - c);
      if (analysis) analysis[band * taps + n] = 2.0 * p[n] * std::cos(theta + phase);
      if (synthesis) synthesis[band * taps + n] = 2.0 * p[n] * std::cos(theta - phase);
    }
  }
  if (cutoff) *cutoff = wc;
  return CC_OK;
}

extern "C" cc_status cc_pqmf_layer_weights(int32_t bands, int32_t taps, double beta, float* analysis_conv,
                                           float* synthesis_convt) {
  if (bands < 2 || taps < 2 || beta < 0.0) return cc::fail(CC_ERR_INVALID_ARG, "bad PQMF size");
  std::vector<double> g((size_t)bands * taps);
  const cc_status s = cc_pqmf_design(bands, taps, beta, nullptr, g.data(), nullptr);
  if (s) return s;
  for (size_t i = 0; i < g.size(); ++i) {
    if (analysis_conv) analysis_conv[i] = (float)g[i];
    if (synthesis_convt) synthesis_convt[i] = (float)(bands * g[i]);
  }
  return CC_OK;
}
