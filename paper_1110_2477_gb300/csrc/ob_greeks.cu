// ob_greeks.cu -- the follow-up launches of the adjoint (Greeks) with larger slices.
#include "ob_kern.cuh"

namespace obl {

__global__ void __launch_bounds__(kTeamBlock, 1) k_greeks_retry(
    const obk::Opt* __restrict__ opts, double* out, double* grad, int* status, char* arena,
    size_t cta_bytes, const int* in_count, const int* in_list, int* head, int* ovf_count, int* ovf_list,
    int last) {
  __shared__ long long tbuf[obk::BlockTeam<kNW>::BUF];
  obk::BlockTeam<kNW> bt{tbuf};
  char* my = arena + (size_t)blockIdx.x * cta_bytes;
  const int cnt = *((volatile const int*)in_count);
  for (;;) {
    int v = 0;
    if (threadIdx.x == 0) v = atomicAdd(head, 1);
    const int idx = bt.bcast0(v);
    if (idx >= cnt) break;
    const int oi = in_list[idx];
    const obk::Opt o = opts[oi];
    int rc;
    double ask, bid, gA[obk::NPAR], gB[obk::NPAR];
    greeks_one(bt, o, my, cta_bytes, rc, ask, bid, gA, gB, false);
    if (threadIdx.x == 0) greeks_finish(oi, rc, ask, bid, gA, gB, out, grad, status, ovf_count, ovf_list, !last);
    bt.sync();
  }
}

cudaError_t launch_greeks_retry(int grid, cudaStream_t s, const obk::Opt* opts, double* out, double* grad,
                                int* status, char* arena, size_t cta_bytes, const int* in_count,
                                const int* in_list, int* head, int* ovf_count, int* ovf_list, int last) {
  k_greeks_retry<<<grid, kTeamBlock, 0, s>>>(opts, out, grad, status, arena, cta_bytes, in_count, in_list, head,
                                             ovf_count, ovf_list, last);
  return cudaGetLastError();
}

}  // namespace obl
