// ob_path.cu -- the kernel and launch of the hedge along a path (ob_path.cuh): one 16-warp
// CTA team per option from a device queue, and a follow-up launch for the options that
// outgrow their slice.
#include "ob_kern.cuh"
#include "ob_path.cuh"

namespace obl {

// One 16-warp CTA team per option, taken from a device queue: position q = atomicAdd(head)
// of order (the costliest first; index order when order is null), q < n, or q < *n_dev when
// n_dev is set (a follow-up launch reads the count its predecessor left).  With ovf_count
// set, an option that outgrows its slice is appended to ovf_list for the follow-up launch
// and its results are left to it; without, it gets ST_CAPACITY and NaN.
__global__ void __launch_bounds__(512, 1) k_tc_path(const obk::Opt* __restrict__ opts, int n,
                                                    const int* n_dev, const int* order, int* head,
                                                    const int8_t* __restrict__ moves, long long stride,
                                                    double* out, double* hold, double* cash, int* stop,
                                                    int* status, char* arena, size_t cta_bytes,
                                                    int* ovf_count, int* ovf_list) {
  __shared__ long long tbuf[obk::BlockTeam<16>::BUF];
  __shared__ int s_next;
  obk::BlockTeam<16> bt{tbuf};
  char* my = arena + (size_t)blockIdx.x * cta_bytes;
  const int count = n_dev ? *n_dev : n;
  for (;;) {
    if (threadIdx.x == 0) {
      const int q = atomicAdd(head, 1);
      s_next = q < count ? (order ? order[q] : q) : -1;
    }
    __syncthreads();
    const int i = s_next;
    if (i < 0) break;
    const obk::Opt o = opts[i];
    double* h = hold + 2 * (stride + 1) * (long long)i;
    double* c = cash ? cash + 2 * (stride + 1) * (long long)i : nullptr;
    double ask, bid;
    int st = -1, rc;
    if (o.N > stride) {
      rc = obk::ST_ARG;
      ask = bid = dnan();
    } else {
      rc = check_option(o, true);
      ask = bid = dnan();
      if (rc == obk::ST_OK)
        rc = obk::path_one(bt, o, moves + stride * (long long)i, my, cta_bytes, ask, bid, h, c, st);
    }
    if (rc == obk::ST_CAPACITY && ovf_count) {  // to the follow-up launch, with more scratch
      if (threadIdx.x == 0) ovf_list[atomicAdd(ovf_count, 1)] = i;
      __syncthreads();
      continue;
    }
    if (threadIdx.x == 0) {
      out[2 * i] = rc ? dnan() : ask;
      out[2 * i + 1] = rc ? dnan() : bid;
      stop[i] = rc ? -1 : st;
      if (status) status[i] = rc;
    }
    const long long first = rc ? 0 : 2 * ((long long)o.N + 1);
    for (long long k = first + threadIdx.x; k < 2 * (stride + 1); k += blockDim.x) {
      h[k] = dnan();
      if (c) c[k] = dnan();
    }
    __syncthreads();
  }
}

cudaError_t launch_path(int grid, cudaStream_t s, const obk::Opt* opts, int n, const int* n_dev, const int* order,
                        int* head, const int8_t* moves, long long stride, double* out, double* hold, double* cash,
                        int* stop, int* status, char* arena, size_t cta_bytes, int* ovf_count, int* ovf_list) {
  k_tc_path<<<grid, 512, 0, s>>>(opts, n, n_dev, order, head, moves, stride, out, hold, cash, stop, status, arena,
                                 cta_bytes, ovf_count, ovf_list);
  return cudaGetLastError();
}

}  // namespace obl
