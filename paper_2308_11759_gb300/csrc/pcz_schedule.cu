// pcz_schedule.cu -- the tolerance schedules of Sec. 5.1 and the lossless
// sweep of Sec. 5.1.3 behind the C ABI (host code; the range reduction and
// the compression they call run in the library's kernels).
//
// Sec. 5.1 measures every tolerance relative to tau_0, the range of the field
// values, and lowers it geometrically from component to component: tau_i =
// 2^(-Delta i) tau_0 for the binary schedules of the experiments.  The decade
// schedule tau_i = 10^-(first + i - 1) tau_0 is the same rule with a factor
// of ten per component.  Everything is computed in double on the host, once:
// the kernels only ever see the finished tolerances.
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "pcz_host.h"

namespace {

// 2^-k as a double (0 below the smallest subnormal), exact
double exp2_neg(int k) { return k > 1074 ? 0.0 : std::ldexp(1.0, -k); }

// The double nearest 10^-e: the decimal literal "1e-e" read with correct
// rounding (strtod rounds to nearest on every C library this builds with).
double decade(int e) {
  char buf[16];
  std::snprintf(buf, sizeof buf, "1e-%d", e);
  return std::strtod(buf, nullptr);
}

}  // namespace

extern "C" {

pc_status pc_tau_schedule(pc_tau_kind kind, double tau0, int param, int n, double* tau) {
  if (!tau || n < 1 || n > PC_MAX_COMPONENTS) return pcz::api_fail(PC_ERR_ARG, "bad n or NULL output");
  if (!(tau0 > 0.0) || !std::isfinite(tau0)) return pcz::api_fail(PC_ERR_ARG, "tau_0 must be positive and finite");
  if (kind == PC_TAU_BINARY) {
    if (param < 1 || (long long)param * n > 4096) return pcz::api_fail(PC_ERR_ARG, "Delta must be in 1..4096/n");
    for (int i = 1; i <= n; ++i) tau[i - 1] = tau0 * exp2_neg(param * i);  // one rounding
  } else if (kind == PC_TAU_DECADE) {
    if (param < 0 || param + n - 1 > 400) return pcz::api_fail(PC_ERR_ARG, "decade exponents must be in 0..400");
    for (int i = 1; i <= n; ++i) tau[i - 1] = decade(param + i - 1) * tau0;  // one rounding
  } else {
    return pcz::api_fail(PC_ERR_ARG, "unknown schedule kind");
  }
  return PC_OK;
}

pc_status pc_field_tau_schedule(const void* field, int64_t count, pc_dtype dtype, pc_tau_kind kind, int param, int n,
                                void* cuda_stream, double* tau) {
  pcz::TraceRange trace_("pc_field_tau_schedule");
  double lo = 0.0, hi = 0.0;
  const pc_status st = pc_field_range(field, count, dtype, cuda_stream, &lo, &hi);
  if (st != PC_OK) return st;
  const double tau0 = hi - lo;  // Sec. 5.1: tau_0 = max - min, one rounding in double
  if (!(tau0 > 0.0)) return pcz::api_fail(PC_ERR_ARG, "the field is constant: its range is 0");
  if (!std::isfinite(tau0)) return pcz::api_fail(PC_ERR_ARG, "the range of the field overflows a double");
  return pc_tau_schedule(kind, tau0, param, n, tau);
}

pc_status pc_lossless_sweep(const void* field, const int64_t* dims, int ndims, pc_dtype dtype, int delta, int n_max,
                            void* cuda_stream, pc_streams** out, int* k, double* bits_per_value) {
  pcz::TraceRange trace_("pc_lossless_sweep");
  if (!out || !k || !bits_per_value || !dims || ndims < 1 || ndims > 3)
    return pcz::api_fail(PC_ERR_ARG, "bad arguments");
  *out = nullptr;
  *k = 0;
  *bits_per_value = 0.0;
  if (n_max < 1 || n_max > PC_MAX_COMPONENTS) return pcz::api_fail(PC_ERR_ARG, "n_max must be in 1..64");
  if (delta < 1 || delta > 64) return pcz::api_fail(PC_ERR_ARG, "delta must be in 1..64");
  int64_t count = 1;
  for (int a = 0; a < ndims; ++a) {
    if (dims[a] < 1) return pcz::api_fail(PC_ERR_ARG, "extents must be positive");
    count *= dims[a];
  }
  double lo = 0.0, hi = 0.0;
  pc_status st = pc_field_range(field, count, dtype, cuda_stream, &lo, &hi);
  if (st != PC_OK) return st;
  // tau_0: the range; a constant field has none, and its own magnitude (at
  // least 1) stands in for it
  double tau0 = hi - lo;
  if (!(tau0 > 0.0)) tau0 = std::fmax(std::fabs(lo), 1.0);
  if (!std::isfinite(tau0)) return pcz::api_fail(PC_ERR_ARG, "the range of the field overflows a double");
  double tau[PC_MAX_COMPONENTS];
  int n = 0;
  for (int i = 1; i <= n_max; ++i) {  // the schedule's positive part
    const double t = tau0 * exp2_neg(delta * i);
    if (!(t > 0.0) || (n && !(t < tau[n - 1]))) break;
    tau[n++] = t;
  }
  if (n == 0) return pcz::api_fail(PC_ERR_ARG, "no positive tolerance in the schedule");
  pc_streams* s = nullptr;
  st = pc_compress(field, dims, ndims, dtype, tau, n, cuda_stream, &s);
  if (st != PC_OK) return st;
  // the first component whose computed tolerance (Sec. 4.3) is 0 reproduces x
  uint64_t bits = 0;
  for (int i = 0; i < n; ++i) {
    bits += s->words[i] * 64 + (uint64_t)s->nchunks * 8 * 8 + (uint64_t)s->nbricks * 2 * 8;
    if (s->measured[i] == 0.0) {
      *k = i + 1;
      *bits_per_value = (double)bits / (double)count;
      break;
    }
  }
  *out = s;
  return PC_OK;
}

}  // extern "C"
