// transport_f32.cu -- production (float) instantiation of the photon-history
// kernel; see transport.cuh.
#include "transport.cuh"

namespace mcs {
void compute_coefficients(const TransportSetup &ts, std::vector<double> &cd, std::vector<float> &cf,
                          std::vector<float> &sig_tab) {
  host_coefficients(ts, cd, cf);
  host_sigma_table(ts, sig_tab);
}
int launch_transport_f32(const TransportSetup &ts, cudaStream_t s) { return launch_transport_t<float>(ts, s); }
int launch_debug_kn_f32(double e, uint64_t seed, uint64_t n, double *c, double *p, cudaStream_t s) {
  return launch_debug_kn_t<float>(e, seed, n, c, p, s);
}
int launch_debug_beam_f32(const TransportSetup &ts, uint64_t n, const double p0[3], const double d[3], double e,
                          unsigned long long *t, cudaStream_t s) {
  return launch_debug_beam_t<float>(ts, n, p0, d, e, t, s);
}
}  // namespace mcs
