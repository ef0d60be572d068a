// Error reporting and the host-side Green-Kubo integral of the C ABI.
#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "common.cuh"

namespace otf {

namespace {
thread_local char g_err[512] = "";
}

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

}  // namespace otf

extern "C" {

const char *md_last_error(void) { return otf::g_err; }

// Trapezoid rule on the readout grid (Sec. 2.3: the Green-Kubo integrals of
// Eqs. (visc) and (therm) up to a maximum lag, by numerical integration).
// The integrand is taken as the straight line between neighbouring points,
// so a cut inside an interval integrates the interpolated line up to t_cut.
int gk_integrate(const double *t, const double *c, int64_t n, double t_cut, double prefactor,
                 double *integral, double *running) {
  otf::clear_error();
  if (!t || !c || !integral || n < 1) {
    otf::set_error("gk_integrate: null argument or n < 1");
    return MD_EINVAL;
  }
  for (int64_t i = 1; i < n; ++i)
    if (!(t[i] > t[i - 1])) {
      otf::set_error("gk_integrate: times must increase (t[%lld] <= t[%lld])", (long long)i,
                     (long long)(i - 1));
      return MD_EINVAL;
    }
  double area = 0.0;    // integral from t[0] to t[i]
  double at_cut = 0.0;  // integral from t[0] to t_cut
  bool cut_found = t_cut <= t[0];
  if (running) running[0] = 0.0;
  for (int64_t i = 0; i + 1 < n; ++i) {
    const double h = t[i + 1] - t[i];
    if (!cut_found && t_cut < t[i + 1]) {
      const double w = t_cut - t[i];
      const double c_cut = c[i] + (c[i + 1] - c[i]) * (w / h);
      at_cut = area + 0.5 * w * (c[i] + c_cut);
      cut_found = true;
    }
    area += 0.5 * h * (c[i] + c[i + 1]);
    if (running) running[i + 1] = prefactor * area;
  }
  *integral = prefactor * (cut_found ? at_cut : area);
  return MD_OK;
}

}  // extern "C"
