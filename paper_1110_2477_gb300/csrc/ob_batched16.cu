// ob_batched16.cu -- the batched kernel for CTA teams of 16 and 12 warps.
#include "ob_kern.cuh"

namespace obl {

#define OB_ARGS a.opts, a.n, a.order, a.out, a.status, a.arena, a.cta_bytes, a.ctl, a.ovf_list, a.ds, a.chip_points, a.hedge

cudaError_t launch_batched_wide(int nw, bool warps, int grid, cudaStream_t s, const BatchedArgs& a) {
  if (nw == 16) {
    if (warps) k_tc_batched<16, true><<<grid, 512, 0, s>>>(OB_ARGS);
    else k_tc_batched<16, false><<<grid, 512, 0, s>>>(OB_ARGS);
  } else if (nw == 12) {
    if (warps) k_tc_batched<12, true><<<grid, 384, 0, s>>>(OB_ARGS);
    else k_tc_batched<12, false><<<grid, 384, 0, s>>>(OB_ARGS);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
#undef OB_ARGS

}  // namespace obl
