// ob_batched8.cu -- the batched kernel for CTA teams of 8 and 4 warps, and the
// instantiations with the fused level step (w on chip) for 16 and 8 warps.
#include "ob_kern.cuh"

namespace obl {

#define OB_ARGS a.opts, a.n, a.order, a.out, a.status, a.arena, a.cta_bytes, a.ctl, a.ovf_list, a.ds, a.chip_points, a.hedge

cudaError_t launch_batched_narrow(int nw, bool warps, bool chip, int grid, size_t smem, cudaStream_t s,
                                  const BatchedArgs& a) {
  if (chip) {
    if (nw == 16) k_tc_batched<16, false, true><<<grid, 512, smem, s>>>(OB_ARGS);
    else if (nw == 8) k_tc_batched<8, false, true><<<grid, 256, smem, s>>>(OB_ARGS);
    else return cudaErrorInvalidValue;
  } else if (nw == 8) {
    if (warps) k_tc_batched<8, true><<<grid, 256, 0, s>>>(OB_ARGS);
    else k_tc_batched<8, false><<<grid, 256, 0, s>>>(OB_ARGS);
  } else if (nw == 4) {
    if (warps) k_tc_batched<4, true><<<grid, 128, 0, s>>>(OB_ARGS);
    else k_tc_batched<4, false><<<grid, 128, 0, s>>>(OB_ARGS);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
#undef OB_ARGS

cudaError_t set_chip_smem(int bytes16, int bytes8) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_batched<16, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       bytes16);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tc_batched<8, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes8);
}

}  // namespace obl
