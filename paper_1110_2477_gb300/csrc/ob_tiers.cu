// ob_tiers.cu -- the follow-up launches of the batched form (larger slices for options
// that outgrew theirs) and the plain one-warp-per-option kernel.
#include "ob_kern.cuh"

namespace obl {

// Follow-up launch: the options of in_list (count at *in_count), one per CTA,
// with larger slices.
__global__ void __launch_bounds__(kTeamBlock, 2) k_tc_retry(
    const obk::Opt* __restrict__ opts, double* out, int* status, char* arena, size_t cta_bytes,
    const int* in_count, const int* in_list, int* head, int* ovf_count, int* ovf_list, int last,
    DevStats* ds, double* hedge) {
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
    double ask, bid;
    obk::Stats st;
    price_one(bt, o, my, cta_bytes, rc, ask, bid, st);
    if (threadIdx.x == 0) finish(oi, rc, ask, bid, st, o, out, status, ovf_count, ovf_list, !last, ds, hedge);
    bt.sync();
  }
}

// Plain form: one warp per option, static assignment in index order, no retry.
__global__ void __launch_bounds__(kBlock) k_tc_plain(const obk::Opt* __restrict__ opts, int n,
                                                     double* out, int* status, char* arena,
                                                     size_t wbytes, int nworkers, DevStats* ds) {
  obk::WarpTeam tm;
  const int wid = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  if (wid >= nworkers) return;
  char* my = arena + (size_t)wid * wbytes;
  for (int oi = wid; oi < n; oi += nworkers) {
    const obk::Opt o = opts[oi];
    int rc;
    double ask, bid;
    obk::Stats st;
    price_one(tm, o, my, wbytes, rc, ask, bid, st);
    if (tm.lane() == 0) finish(oi, rc, ask, bid, st, o, out, status, nullptr, nullptr, false, ds, nullptr);
    tm.sync();
  }
}

cudaError_t launch_retry(int grid, cudaStream_t s, const obk::Opt* opts, double* out, int* status, char* arena,
                         size_t cta_bytes, const int* in_count, const int* in_list, int* head, int* ovf_count,
                         int* ovf_list, int last, DevStats* ds, double* hedge) {
  k_tc_retry<<<grid, kTeamBlock, 0, s>>>(opts, out, status, arena, cta_bytes, in_count, in_list, head, ovf_count,
                                         ovf_list, last, ds, hedge);
  return cudaGetLastError();
}

cudaError_t launch_plain(int blocks, cudaStream_t s, const obk::Opt* opts, int n, double* out, int* status,
                         char* arena, size_t wbytes, int nworkers, DevStats* ds) {
  k_tc_plain<<<blocks, kBlock, 0, s>>>(opts, n, out, status, arena, wbytes, nworkers, ds);
  return cudaGetLastError();
}

}  // namespace obl
