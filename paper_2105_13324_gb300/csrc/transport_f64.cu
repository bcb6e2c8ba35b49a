// transport_f64.cu -- verification (double) instantiation of the
// photon-history kernel; compiled with --fmad=false so that products and sums
// are rounded one by one, in the order written; see transport.cuh.
#include "transport.cuh"

namespace mcs {
int launch_transport_f64(const TransportSetup &ts, cudaStream_t s) { return launch_transport_t<double>(ts, s); }
int launch_debug_kn_f64(double e, uint64_t seed, uint64_t n, double *c, double *p, cudaStream_t s) {
  return launch_debug_kn_t<double>(e, seed, n, c, p, s);
}
int launch_debug_beam_f64(const TransportSetup &ts, uint64_t n, const double p0[3], const double d[3], double e,
                          unsigned long long *t, cudaStream_t s) {
  return launch_debug_beam_t<double>(ts, n, p0, d, e, t, s);
}
}  // namespace mcs
