// ob_batched_half.cu -- the batched kernel whose 16-warp CTAs split into two 8-warp
// teams once the costliest options are taken.
#include "ob_kern.cuh"

namespace obl {

cudaError_t launch_batched_halves(int grid, cudaStream_t s, const BatchedArgs& a) {
  k_tc_batched<16, false, false, true><<<grid, 512, 0, s>>>(a.opts, a.n, a.order, a.out, a.status, a.arena,
                                                            a.cta_bytes, a.ctl, a.ovf_list, a.ds,
                                                            a.chip_points, a.hedge);
  return cudaGetLastError();
}

}  // namespace obl
