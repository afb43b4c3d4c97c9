// ob_greeks8.cu -- the adjoint (Greeks) on 8- and 16-warp CTA teams.
#include "ob_kern.cuh"

namespace obl {

cudaError_t launch_greeks_team8(int grid, cudaStream_t s, const obk::Opt* opts, int n, double* out, double* grad,
                                int* status, char* arena, size_t cta_bytes, int* ctl, int* ovf_list, int allow_full) {
  k_greeks_team<8><<<grid, 256, 0, s>>>(opts, n, out, grad, status, arena, cta_bytes, ctl, ovf_list, allow_full);
  return cudaGetLastError();
}

cudaError_t launch_greeks_team16(int grid, cudaStream_t s, const obk::Opt* opts, int n, double* out, double* grad,
                                 int* status, char* arena, size_t cta_bytes, int* ctl, int* ovf_list, int allow_full) {
  k_greeks_team<16><<<grid, 512, 0, s>>>(opts, n, out, grad, status, arena, cta_bytes, ctl, ovf_list, allow_full);
  return cudaGetLastError();
}

}  // namespace obl
