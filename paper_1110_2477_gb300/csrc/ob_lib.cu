// ob_lib.cu -- the host side of the C ABI declared in include/ob.h (scratch pool,
// call ordering, CUDA graphs, entry points) and the small kernels:
//  k_order        one CTA sorts the option indices by predicted cost (largest first)
//  k_crr          persistent warps: plain CRR recursion without costs, the level kept in
//                 shared memory and updated in place
//  k_gather, k_fp64_probe   the autotuner's sample; the FP64 throughput probe
// The induction kernels live in their own translation units (compiled in parallel):
//  ob_batched16.cu, ob_batched8.cu   k_tc_batched: persistent CTAs take options from a
//                 device queue and run the piecewise-linear induction (ob_tc.cuh) on a
//                 whole-CTA team in their slice of the scratch pool; an option that
//                 outgrows its slice goes to an overflow list
//  ob_tiers.cu    k_tc_retry (the follow-up launches: 16 CTAs, then one, larger slices)
//                 and k_tc_plain (one warp per option in index order)
//  ob_group.cu    k_tc_group: cooperative launches of a CTA per SM, each option in
//                 turn, every level split over all CTAs (TcGroup) or, for light levels of
//                 options with even columns, trapezoid rounds of levels (TcTrap); bounded
//                 grid barriers
//  ob_greeks8.cu, ob_greeks.cu   the adjoint (ob_adj.cuh) on CTA teams, single warps,
//                 and its follow-up launches
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "ob_kern.cuh"

using namespace obl;

namespace {

// Bitonic sort of (cost, index) keys, descending, in one CTA; also decides how
// many of the costliest options go to whole-CTA teams (ctl[C_NHEAVY]).
__global__ void k_order(const obk::Opt* __restrict__ opts, int n, int npad, int* __restrict__ order,
                        int* ctl, int nwarps, int nctas, double heavy_factor) {
  extern __shared__ unsigned long long keys[];
  __shared__ double part[32];
  double mysum = 0.0;
  for (int i = threadIdx.x; i < npad; i += blockDim.x) {
    unsigned long long key = 0;
    if (i < n) {
      const double c = predicted_cost(opts[i]);
      mysum += c;
      key = ((unsigned long long)c + 1ULL) << 20 | (unsigned long long)i;
    }
    keys[i] = key;
  }
  for (int d = 16; d >= 1; d >>= 1) mysum += __shfl_down_sync(0xffffffffu, mysum, d);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = mysum;
  __syncthreads();
  for (int size = 2; size <= npad; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < npad; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool desc = (i & size) == 0;
          const unsigned long long a = keys[i], b = keys[j];
          if ((a < b) == desc) { keys[i] = b; keys[j] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) order[i] = (int)(keys[i] & 0xFFFFF);
  if (threadIdx.x == 0) {
    double total = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += part[w];
    int nh = 0;
    if (n <= nctas) {
      nh = n;  // few options: every option gets a whole CTA
    } else {
      const double thr = heavy_factor * total / (double)nwarps;
      while (nh < n && (double)(keys[nh] >> 20) > thr) ++nh;
    }
    ctl[C_NHEAVY] = nh;
  }
}

// ------------------------------------------------------------------ plain CRR
// c_{t,j} = max(P_{t,j}, pu c_{t+1,j+1} + pd c_{t+1,j}), pu = p/r, pd = (1-p)/r;
// P is tabulated per option by stock exponent e = 2j - t (max(payoff, 0)).
// Lanes take interleaved nodes so that shared-memory and table accesses are
// unit-stride; the up-successor value comes from the neighbour lane.

__global__ void __launch_bounds__(kBlock) k_crr(const obk::Opt* __restrict__ opts, int n, double* out,
                                                int* status, char* arena, size_t wbytes, int nworkers,
                                                int* ctl) {
  extern __shared__ double crr_sm[];
  obk::WarpTeam tm;
  const int lane = tm.lane();
  const int wid = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  if (wid >= nworkers) return;
  double* mysm = crr_sm + (size_t)(threadIdx.x >> 5) * kCrrSmem;
  char* my = arena + (size_t)wid * wbytes;
  for (;;) {
    int v = 0;
    if (lane == 0) v = atomicAdd(&ctl[0], 1);
    const int oi = tm.bcast0(v);
    if (oi >= n) break;
    const obk::Opt o = opts[oi];
    int rc = check_option(o, false);
    double res = dnan();
    if (rc == obk::ST_OK) {
      const int N = o.N;
      const double dt = o.T / N;
      const double u = exp(o.sigma * sqrt(dt));
      const double d = 1.0 / u;
      const double r = exp(o.R * dt);
      const size_t ptab_bytes = obk::al256(sizeof(double) * (2 * (size_t)N + 1));
      const bool in_smem = (N + 2) <= kCrrSmem;
      const size_t need = ptab_bytes + (in_smem ? 0 : sizeof(double) * ((size_t)N + 2));
      if (!(d < r && r < u)) {
        rc = obk::ST_ARBITRAGE;
      } else if (need > wbytes) {
        rc = obk::ST_CAPACITY;
      } else {
        const double p = (r - d) / (u - d);
        const double pu = p / r, pd = (1.0 - p) / r;
        double* P = (double*)my;  // P[e + N], e = -N..N
        double* V = in_smem ? mysm : (double*)(my + ptab_bytes);
        for (int e = lane; e <= 2 * N; e += 32) P[e] = crr_payoff(o, o.S0 * pow(u, (double)(e - N)));
        tm.sync();
        for (int j = lane; j <= N; j += 32) V[j] = P[2 * j];
        tm.sync();
        for (int t = N - 1; t >= 0; --t) {
          const int width = t + 1;  // nodes of level t; level t+1 holds width+1 values
          const double* Pt = P + (N - t);
          for (int base = 0; base < width; base += 32) {
            const int i = base + lane;
            const double cur = (i <= width) ? V[i] : 0.0;
            double up = __shfl_down_sync(0xffffffffu, cur, 1);
            const double extra = (base + 32 <= width) ? V[base + 32] : 0.0;
            if (lane == 31) up = extra;
            tm.sync();
            if (i < width) {
              V[i] = crr_step(pu, pd, up, cur, Pt[2 * i]);
            }
            tm.sync();
          }
        }
        res = V[0];
        tm.sync();
      }
    }
    if (lane == 0) {
      out[oi] = res;
      if (status) status[oi] = rc;
    }
  }
}

// ------------------------------------------------------------------ FP64 throughput probe
// Each thread runs kProbeChains independent chains of a = a * b + c (one DFMA each),
// so the FP64 pipe, not latency, bounds the loop; the result is written so that the
// compiler keeps every chain.  2 flops per DFMA.
constexpr int kProbeChains = 8;
__global__ void __launch_bounds__(256) k_fp64_probe(long long iters, double b, double c, double* sink) {
  double a[kProbeChains];
  for (int i = 0; i < kProbeChains; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) a[i] = fma(a[i], b, c);
  }
  double t = 0.0;
  for (int i = 0; i < kProbeChains; ++i) t += a[i];
  if (t == 12345.678) sink[0] = t;  // never true for b, c near 1 and 0
}

// Every stride-th option, for the autotuner's sample.
__global__ void k_gather(const obk::Opt* __restrict__ src, int n, int stride, int m, obk::Opt* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    const long long j = (long long)i * stride;
    dst[i] = src[j < n ? j : n - 1];
  }
}

// ------------------------------------------------------------------ host side
thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s", cudaGetErrorString(e));
  return OB_ERR_CUDA;
}

// One instantiated CUDA graph of the batched launch sequence, keyed by the call's
// pointers, size and team width (a replay reads the buffers' current contents).
struct GraphEntry {
  const void* params = nullptr;
  void* out = nullptr;
  void* status = nullptr;
  int n = 0;
  int team_warps = 0;
  int chip = 0;
  double split = 0.0;
  const double* hedge = nullptr;
  cudaGraphExec_t exec = nullptr;
};
constexpr int kGraphCache = 4;
constexpr int kTuneCands = 7;  // configurations the autotuner times

// Scratch budgets.  The pool is one device allocation that grows to the largest
// need of any call so far (never shrinks before ob_release); OB_POOL_MB fixes its size.
constexpr size_t kMinArena = 1ull << 30;          // smallest pool (room for the retry tiers)
constexpr size_t kPlainWarpBytes = 8ull << 20;    // per warp of the one-warp-per-option form
constexpr size_t kCrrWarpBytes = 512ull << 10;    // per warp of the CRR kernel
constexpr size_t kGreeksSmBytes = 128ull << 20;   // per SM of the Greeks form (level store)

struct DevPool {
  bool init = false;
  int sms = 0;
  int warps_per_sm = 16;
  size_t sm_bytes = 32ull << 20;  // first-tier scratch per SM of the batched form
  int smem_sm = 0;                // shared memory per SM and the largest per CTA (bytes)
  int smem_cta = 0;
  int chip_req = 0;               // on-chip w points per CTA (-1 all that fit, 0 off; OB_CHIP_POINTS)
  size_t fixed_bytes = 0;         // OB_POOL_MB: the pool has exactly this size
  double heavy_factor = kHeavyFactor;
  double split_factor = kSplitFactor;  // 16-warp CTAs: options below it go to half-CTA teams
  int team_warps = 16;  // whole-SM teams: one 512-thread CTA per SM
  int greeks_warps = 16; // warps of a Greeks CTA team (16 or 8)
  int greeks_full = 1;   // records of every level when they fit (OB_GREEKS_FULL=0: checkpoints only)
  size_t path_bytes = kGreeksSmBytes;  // first-tier scratch per CTA of the path form (OB_PATH_MB)
  char* arena = nullptr;
  size_t arena_bytes = 0;
  int* ctl = nullptr;      // 2 ints per tier (queue head, overflow count)
  int* order = nullptr;    // kSortMax
  int* lists = nullptr;    // 2 overflow lists of list_cap
  size_t list_cap = 0;
  DevStats* stats = nullptr;
  // host-buffer entry point
  cudaStream_t hstream = nullptr;
  ob_option_t* hparams = nullptr;
  double* hout = nullptr;
  int* hstatus = nullptr;
  size_t hcap = 0;
  int last_tiers = 0;
  // CUDA graphs of the batched form
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;
  GraphEntry graphs[kGraphCache];
  int graph_next = 0;
  int last_graph = 0;  // 0 direct launches, 1 captured now, 2 replayed
  GroupState* gstate = nullptr;  // whole-GPU form
  int group_ctas = 0;
  unsigned long long wide_wait_ns = kGroupWaitNs;  // bound of one grid-barrier wait
  double wide_split_x = kWideSplitX;  // whole-GPU form: nodes split above this (OB_WIDE_SPLIT_X)
  int test_skip_calls = 0;  // OB_TEST_WIDE_SKIP: calls in which one CTA never arrives
  // autotuner sample buffers
  obk::Opt* tune_params = nullptr;
  double* tune_out = nullptr;
  int* tune_status = nullptr;
  int tune_cap = 0;
  // ordering of calls: each call's work waits for the previous call's on the device
  cudaEvent_t order_ev = nullptr;
  bool order_valid = false;
};

std::mutex g_mu;
std::mutex g_graph_mu;
std::mutex g_call_mu[64];  // one enqueue at a time per device
std::mutex g_host_mu[64];  // one host-buffer call at a time per device
DevPool g_pool[64];

size_t env_size(const char* name, size_t dflt) {
  const char* s = getenv(name);
  if (!s || !*s) return dflt;
  const long long v = atoll(s);
  return v > 0 ? (size_t)v : dflt;
}

void drop_graphs(DevPool* P);

// Dynamic shared memory a CTA of NW warps can take for the on-chip w arrays: its share
// of the SM (16 / NW CTAs per SM; 1 KiB per CTA is reserved by the system) less the
// team's exchange area, capped by the per-CTA limit.
int chip_smem_cap(int smem_sm, int smem_cta, int nw) {
  const int per_sm = 16 / nw;
  int b = smem_sm / per_sm - 1024 - (int)sizeof(long long) * 2 * (32 * nw + 4 * nw + 8);
  const int lim = smem_cta - (int)sizeof(long long) * 2 * (32 * nw + 4 * nw + 8);
  if (b > lim) b = lim;
  return b > 0 ? b & ~255 : 0;
}

// Points of the on-chip w arrays for teams of nw warps (0: the fused step is off).
int chip_points(const DevPool* P, int nw) {
  const int fit = chip_smem_cap(P->smem_sm, P->smem_cta, nw) / obk::WBUF_POINT_BYTES;
  if (P->chip_req < 0) return fit;
  return P->chip_req < fit ? P->chip_req : fit;
}

// The pool of the current device, initialised on first use (no scratch yet).
int pool_get(DevPool** out, int* dev_out = nullptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= 64) return OB_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  DevPool& P = g_pool[dev];
  if (!P.init) {
    e = cudaDeviceGetAttribute(&P.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e);
    P.warps_per_sm = (int)env_size("OB_WARPS_PER_SM", 16);
    P.sm_bytes = (env_size("OB_ARENA_MB", 2) << 20) * 16;  // OB_ARENA_MB: MiB per warp slot
    if (const size_t kb = env_size("OB_SM_KB", 0)) P.sm_bytes = kb << 10;  // or KiB per SM
    P.fixed_bytes = env_size("OB_POOL_MB", 0) << 20;
    if (const char* hf = getenv("OB_HEAVY_FACTOR")) P.heavy_factor = atof(hf);
    if (const char* sf = getenv("OB_SPLIT_FACTOR")) P.split_factor = atof(sf);
    if (const char* tw = getenv("OB_TEAM_WARPS")) {
      const int v = atoi(tw);
      if (v == 4 || v == 8 || v == 12 || v == 16) P.team_warps = v;
    }
    if (const char* g = getenv("OB_GRAPH")) P.use_graphs = atoi(g) != 0;
    if (const char* g = getenv("OB_GREEKS_WARPS")) P.greeks_warps = atoi(g) == 8 ? 8 : 16;
    if (const char* g = getenv("OB_GREEKS_FULL")) P.greeks_full = atoi(g) != 0;
    P.path_bytes = env_size("OB_PATH_MB", kGreeksSmBytes >> 20) << 20;
    P.wide_wait_ns = env_size("OB_WIDE_WAIT_MS", kGroupWaitNs / 1000000ULL) * 1000000ULL;
    if (const char* x = getenv("OB_WIDE_SPLIT_X")) P.wide_split_x = atof(x);
    P.test_skip_calls = (int)env_size("OB_TEST_WIDE_SKIP", 0);
    if (const char* c = getenv("OB_CHIP_POINTS")) P.chip_req = atoi(c);
    if ((e = cudaDeviceGetAttribute(&P.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) !=
            cudaSuccess ||
        (e = cudaDeviceGetAttribute(&P.smem_cta, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
      return cuda_fail(e);
    if ((e = set_chip_smem(chip_smem_cap(P.smem_sm, P.smem_cta, 16), chip_smem_cap(P.smem_sm, P.smem_cta, 8))) !=
        cudaSuccess)
      return cuda_fail(e);
    if (cudaMalloc(&P.ctl, sizeof(int) * C_WORDS) != cudaSuccess ||
        cudaMalloc(&P.order, sizeof(int) * kSortMax) != cudaSuccess ||
        cudaMalloc(&P.stats, sizeof(DevStats)) != cudaSuccess) {
      cudaGetLastError();
      return OB_ERR_NOMEM;
    }
    cudaMemset(P.stats, 0, sizeof(DevStats));
    if ((e = cudaEventCreateWithFlags(&P.order_ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e);
    e = cudaFuncSetAttribute(k_order, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(unsigned long long) * kSortMax));
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaFuncSetAttribute(k_crr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * kCrrSmem * (kBlock / 32)));
    if (e != cudaSuccess) return cuda_fail(e);
    P.init = true;
  }
  *out = &P;
  if (dev_out) *dev_out = dev;
  return OB_OK;
}

// Make room for a call: overflow lists of need_list entries and a scratch pool of at
// least need_arena bytes (at least kMinArena; exactly OB_POOL_MB when that is set).
// Growing synchronises the device first (work in flight may use the old buffers) and
// drops the cached graphs (they hold the old addresses).  The caller holds g_call_mu.
int pool_reserve(DevPool* P, size_t need_list, size_t need_arena) {
  if (need_arena < kMinArena) need_arena = kMinArena;
  if (P->fixed_bytes) need_arena = P->fixed_bytes;
  const bool grow_list = need_list > P->list_cap;
  const bool grow_arena = P->fixed_bytes ? (P->arena == nullptr) : need_arena > P->arena_bytes;
  if (!grow_list && !grow_arena) return OB_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e);
  drop_graphs(P);
  if (grow_list) {
    cudaFree(P->lists);
    P->lists = nullptr;
    P->list_cap = 0;
    if (cudaMalloc(&P->lists, sizeof(int) * 2 * need_list) != cudaSuccess) {
      cudaGetLastError();
      return OB_ERR_NOMEM;
    }
    P->list_cap = need_list;
  }
  if (grow_arena) {
    cudaFree(P->arena);
    P->arena = nullptr;
    P->arena_bytes = 0;
    if (cudaMalloc(&P->arena, need_arena) != cudaSuccess) {
      cudaGetLastError();
      return OB_ERR_NOMEM;
    }
    P->arena_bytes = need_arena;
  }
  return OB_OK;
}

// Calls on one device are ordered on the GPU in the order they were made: a call's
// first operation waits for the previous call's last one (an event), whatever streams
// they use, so concurrent calls never share the queue words, lists and scratch.  Not
// applied while the caller's stream is being captured into a graph (an event from
// outside the capture cannot be waited on there); such calls are ordered by the caller.
struct CallOrder {
  DevPool* P;
  cudaStream_t s;
  bool on = false;
  int begin() {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_fail(e);
    on = cs == cudaStreamCaptureStatusNone;
    if (on && P->order_valid && (e = cudaStreamWaitEvent(s, P->order_ev, 0)) != cudaSuccess)
      return cuda_fail(e);
    return OB_OK;
  }
  int end() {
    if (!on) return OB_OK;
    cudaError_t e = cudaEventRecord(P->order_ev, s);
    if (e != cudaSuccess) return cuda_fail(e);
    P->order_valid = true;
    return OB_OK;
  }
};

// Scratch of the batched form for a call of n options: the first tier's CTAs and the
// bytes each gets (the per-SM budget split over the CTAs of an SM).
int batched_ctas(const DevPool* P, int n) {
  const int nctas = P->sms * (16 / P->team_warps);
  return n < nctas ? n : nctas;
}
size_t batched_need(const DevPool* P, int n) {
  return (size_t)batched_ctas(P, n) * (P->sm_bytes / (16 / P->team_warps));
}

int enqueue_batched(DevPool* P, const obk::Opt* opts, int n, double* out, int32_t* status,
                    cudaStream_t s, double* hedge = nullptr);
int launch_graph(DevPool* P, const obk::Opt* opts, int n, double* out, int32_t* status,
                 cudaStream_t s, double* hedge = nullptr);

int launch_tc(const ob_option_t* params, int64_t n64, double* out, int32_t* status, void* stream,
              bool plain, double* hedge = nullptr) {
  if (n64 < 0 || n64 > (1 << 30)) return OB_ERR_ARG;
  if (n64 == 0) return OB_OK;
  if (!params || !out) return OB_ERR_ARG;
  const int n = (int)n64;
  DevPool* P = nullptr;
  int dev = 0;
  int rc = pool_get(&P, &dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_call_mu[dev]);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  const obk::Opt* opts = (const obk::Opt*)params;
  if (plain) {
    const int max_workers = P->sms * P->warps_per_sm;
    const int workers = n < max_workers ? n : max_workers;
    if ((rc = pool_reserve(P, 1, (size_t)workers * kPlainWarpBytes))) return rc;
    CallOrder co{P, s};
    if ((rc = co.begin())) return rc;
    if ((e = cudaMemsetAsync(P->stats, 0, sizeof(DevStats), s)) != cudaSuccess) return cuda_fail(e);
    size_t wbytes = P->arena_bytes / (size_t)workers;
    if (wbytes > kPlainWarpBytes) wbytes = kPlainWarpBytes;
    wbytes &= ~(size_t)255;
    const int blocks = (workers * 32 + kBlock - 1) / kBlock;
    if ((e = launch_plain(blocks, s, opts, n, out, status, P->arena, wbytes, workers, P->stats)) != cudaSuccess)
      return cuda_fail(e);
    P->last_tiers = 1;
    P->last_graph = 0;
    return co.end();
  }
  if ((rc = pool_reserve(P, (size_t)n, batched_need(P, n)))) return rc;
  CallOrder co{P, s};
  if ((rc = co.begin())) return rc;
  if (!P->use_graphs) {
    P->last_graph = 0;
    rc = enqueue_batched(P, opts, n, out, status, s, hedge);
  } else {
    rc = launch_graph(P, opts, n, out, status, s, hedge);
  }
  if (rc) return rc;
  return co.end();
}

// The batched launch sequence: reset the queue words and counters, order the options
// by predicted cost, run the persistent kernel, then the two follow-up tiers for
// options that outgrew their scratch.  No host synchronisation, so it can be captured.
// hedge (may be null): the hedge at the root, 4 doubles per option; the fused on-chip step
// keeps no w_0 to read it from, so a call that asks for it runs without that step.
int enqueue_batched(DevPool* P, const obk::Opt* opts, int n, double* out, int32_t* status,
                    cudaStream_t s, double* hedge) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(P->ctl, 0, sizeof(int) * C_WORDS, s)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemsetAsync(P->stats, 0, sizeof(DevStats), s)) != cudaSuccess) return cuda_fail(e);
  const int nctas = batched_ctas(P, n);
  const int* order = nullptr;
  // with a heavy factor of 0 every option goes to a CTA team and the kernel leaves out
  // the warp-team loop (and its registers); without the cost order, warps take them all
  const bool warps = P->heavy_factor > 0.0 || n > kSortMax;
  // the on-chip w arrays of the fused level step (CTA teams of 16 or 8 warps only)
  const int chip = (warps || hedge || (P->team_warps != 16 && P->team_warps != 8)) ? 0 : chip_points(P, P->team_warps);
  // 16-warp CTAs that split into two 8-warp teams for the options whose predicted cost is
  // below split_factor x the mean per SM (the costliest ones keep whole CTAs)
  const bool halves = !warps && chip == 0 && P->team_warps == 16 && P->split_factor > 0.0;
  if (n <= kSortMax) {
    int npad = 1;
    while (npad < n) npad <<= 1;
    k_order<<<1, 1024, sizeof(unsigned long long) * npad, s>>>(
        opts, n, npad, P->order, P->ctl, halves ? nctas : nctas * P->team_warps, nctas,
        halves ? P->split_factor : P->heavy_factor);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    order = P->order;
  }
  size_t cta_bytes = P->arena_bytes / (size_t)nctas;
  if (cta_bytes > P->sm_bytes / (16 / P->team_warps)) cta_bytes = P->sm_bytes / (16 / P->team_warps);
  cta_bytes &= ~(size_t)255;
  int* list0 = P->lists;
  int* list1 = P->lists + P->list_cap;
  const size_t chip_bytes = (size_t)chip * obk::WBUF_POINT_BYTES;
  const BatchedArgs ba{opts, n, order, out, status, P->arena, cta_bytes, P->ctl, list0, P->stats, chip, hedge};
  if (halves)
    e = launch_batched_halves(nctas, s, ba);
  else if (chip > 0 || P->team_warps == 8 || P->team_warps == 4)
    e = launch_batched_narrow(P->team_warps, warps, chip > 0, nctas, chip_bytes, s, ba);
  else
    e = launch_batched_wide(P->team_warps, warps, nctas, s, ba);
  if (e != cudaSuccess) return cuda_fail(e);
  const size_t t1_bytes = (P->arena_bytes / kTier1Ctas) & ~(size_t)255;
  e = launch_retry(kTier1Ctas, s, opts, out, status, P->arena, t1_bytes, &P->ctl[C_T0_OVF], list0,
                   &P->ctl[C_T1_HEAD], &P->ctl[C_T1_OVF], list1, 0, P->stats, hedge);
  if (e != cudaSuccess) return cuda_fail(e);
  e = launch_retry(1, s, opts, out, status, P->arena, P->arena_bytes & ~(size_t)255, &P->ctl[C_T1_OVF], list1,
                   &P->ctl[C_T2_HEAD], &P->ctl[C_T2_OVF], nullptr, 1, P->stats, hedge);
  if (e != cudaSuccess) return cuda_fail(e);
  P->last_tiers = kTiers + (order ? 1 : 0);
  return OB_OK;
}

// Replay the cached graph of this call's key, or capture the sequence on the pool's
// capture stream, instantiate it (evicting the oldest entry) and launch it on s.
int launch_graph(DevPool* P, const obk::Opt* opts, int n, double* out, int32_t* status,
                 cudaStream_t s, double* hedge) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  cudaError_t e;
  for (GraphEntry& g : P->graphs) {
    if (g.exec && g.params == opts && g.n == n && g.out == out && g.status == status &&
        g.team_warps == P->team_warps && g.chip == P->chip_req && g.split == P->split_factor &&
        g.hedge == hedge) {
      if ((e = cudaGraphLaunch(g.exec, s)) != cudaSuccess) return cuda_fail(e);
      P->last_graph = 2;
      P->last_tiers = kTiers + (n <= kSortMax ? 1 : 0);
      return OB_OK;
    }
  }
  if (!P->cap_stream &&
      (e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return cuda_fail(e);
  const int rc = enqueue_batched(P, opts, n, out, status, P->cap_stream, hedge);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(P->cap_stream, &graph);
  if (rc || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc ? rc : cuda_fail(e);
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e);
  GraphEntry& g = P->graphs[P->graph_next];
  P->graph_next = (P->graph_next + 1) % kGraphCache;
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = exec;
  g.params = opts;
  g.n = n;
  g.out = out;
  g.status = status;
  g.team_warps = P->team_warps;
  g.chip = P->chip_req;
  g.split = P->split_factor;
  g.hedge = hedge;
  if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) return cuda_fail(e);
  P->last_graph = 1;
  return OB_OK;
}

void drop_graphs(DevPool* P) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (GraphEntry& g : P->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = GraphEntry();
  }
  P->graph_next = 0;
}

// ------------------------------------------------------------------ fixed-scratch form
// Scratch of ob_price_ask_bid_noalloc: one file-scope device array, so that the
// call needs no allocation at all.  Every device that loads the library holds
// it until the process exits.  Layout: control words and counters, the cost
// order, the retry list, then the workers' slices.
constexpr size_t kNoAllocBytes = OB_NOALLOC_SCRATCH_BYTES;
constexpr int kNoAllocMaxOptions = OB_NOALLOC_MAX_OPTIONS;
constexpr int kNoAllocCtas = 16;
constexpr size_t kNoAllocHead = 4096;  // control words + DevStats
constexpr size_t kNoAllocLists = 2 * sizeof(int) * (size_t)kNoAllocMaxOptions;
static __device__ __align__(256) char ob_noalloc_scratch[kNoAllocBytes];

struct NoAllocDev {
  bool ready = false;
  char* base = nullptr;  // device address of ob_noalloc_scratch on this device
};
NoAllocDev g_noalloc[64];

int noalloc_base(char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= 64) return OB_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  NoAllocDev& D = g_noalloc[dev];
  if (!D.ready) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, ob_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    D.base = (char*)p;
    D.ready = true;
  }
  *out = D.base;
  return OB_OK;
}

}  // namespace

extern "C" {

int ob_price_ask_bid(const ob_option_t* params, int64_t n_options, double* out, int32_t* status,
                     void* stream) {
  return launch_tc(params, n_options, out, status, stream, false);
}

int ob_price_ask_bid_hedge(const ob_option_t* params, int64_t n_options, double* out, int32_t* status,
                           double* hedge, void* stream) {
  if (n_options > 0 && !hedge) return OB_ERR_ARG;
  return launch_tc(params, n_options, out, status, stream, false, hedge);
}

int ob_price_ask_bid_plain(const ob_option_t* params, int64_t n_options, double* out,
                           int32_t* status, void* stream) {
  return launch_tc(params, n_options, out, status, stream, true);
}

int ob_price_ask_bid_wide(const ob_option_t* params, int64_t n_options, double* out,
                          int32_t* status, void* stream) {
  if (n_options < 0 || n_options > (1 << 30)) return OB_ERR_ARG;
  if (n_options == 0) return OB_OK;
  if (!params || !out) return OB_ERR_ARG;
  DevPool* P = nullptr;
  int dev = 0;
  int rc = pool_get(&P, &dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_call_mu[dev]);
  cudaError_t e;
  if (!P->gstate) {
    int per_sm = 0, coop = 0;
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess)
      return cuda_fail(e);
    if (!coop) return OB_ERR_CUDA;
    if ((e = group_occupancy(&per_sm)) != cudaSuccess) return cuda_fail(e);
    if (per_sm < 1) return OB_ERR_CUDA;
    int G = P->sms;  // one CTA per SM
    if (G > kGroupMax) G = kGroupMax;
    if (cudaMalloc(&P->gstate, sizeof(GroupState)) != cudaSuccess) {
      cudaGetLastError();
      return OB_ERR_NOMEM;
    }
    P->group_ctas = G;
  }
  if ((rc = pool_reserve(P, 1, (size_t)P->sms * P->sm_bytes))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CallOrder co{P, s};
  if ((rc = co.begin())) return rc;
  if ((e = cudaMemsetAsync(P->gstate, 0, sizeof(GroupState), s)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemsetAsync(P->stats, 0, sizeof(DevStats), s)) != cudaSuccess) return cuda_fail(e);
  const int G = P->group_ctas;
  const size_t shared_bytes = (P->arena_bytes / 8) & ~(size_t)255;
  const size_t cta_bytes = ((P->arena_bytes - shared_bytes) / (size_t)G) & ~(size_t)255;
  const obk::Opt* opts = (const obk::Opt*)params;
  int n = (int)n_options;
  char* arena = P->arena;
  GroupState* gs = P->gstate;
  DevStats* ds = P->stats;
  unsigned long long wait_ns = P->wide_wait_ns;
  int skip_cta = -1;
  if (P->test_skip_calls > 0) {
    --P->test_skip_calls;
    skip_cta = G - 1;
  }
  if ((e = launch_group(G, s, opts, n, out, status, arena, shared_bytes, cta_bytes, gs, ds, wait_ns, skip_cta,
                        P->wide_split_x)) !=
      cudaSuccess)
    return cuda_fail(e);
  P->last_tiers = 1;
  P->last_graph = 0;
  return co.end();
}

int ob_crr_american(const ob_option_t* params, int64_t n_options, double* out, int32_t* status,
                    void* stream) {
  if (n_options < 0 || n_options > (1 << 30)) return OB_ERR_ARG;
  if (n_options == 0) return OB_OK;
  if (!params || !out) return OB_ERR_ARG;
  const int n = (int)n_options;
  DevPool* P = nullptr;
  int dev = 0;
  int rc = pool_get(&P, &dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_call_mu[dev]);
  const int max_workers = P->sms * 12;  // 3 CTAs of 4 warps per SM fit the shared memory
  const int workers = n < max_workers ? n : max_workers;
  if ((rc = pool_reserve(P, 1, (size_t)workers * kCrrWarpBytes))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CallOrder co{P, s};
  if ((rc = co.begin())) return rc;
  cudaError_t e;
  if ((e = cudaMemsetAsync(P->ctl, 0, sizeof(int) * C_WORDS, s)) != cudaSuccess) return cuda_fail(e);
  size_t wbytes = P->arena_bytes / (size_t)workers;
  if (wbytes > kCrrWarpBytes) wbytes = kCrrWarpBytes;
  wbytes &= ~(size_t)255;
  const int blocks = (workers * 32 + kBlock - 1) / kBlock;
  k_crr<<<blocks, kBlock, sizeof(double) * kCrrSmem * (kBlock / 32), s>>>(
      (const obk::Opt*)params, n, out, status, P->arena, wbytes, workers, P->ctl);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
  return co.end();
}

int ob_crr_american_wide(const ob_option_t* params, int64_t n_options, double* out, int32_t* status,
                         void* stream) {
  if (n_options < 0 || n_options > (1 << 30)) return OB_ERR_ARG;
  if (n_options == 0) return OB_OK;
  if (!params || !out) return OB_ERR_ARG;
  DevPool* P = nullptr;
  int dev = 0;
  int rc = pool_get(&P, &dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_call_mu[dev]);
  cudaError_t e;
  if (!P->gstate) {
    if (cudaMalloc(&P->gstate, sizeof(GroupState)) != cudaSuccess) {
      cudaGetLastError();
      return OB_ERR_NOMEM;
    }
  }
  int per_sm = 0, coop = 0;
  if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return cuda_fail(e);
  if (!coop) return OB_ERR_CUDA;
  if ((e = crr_group_occupancy(&per_sm)) != cudaSuccess) return cuda_fail(e);
  if (per_sm < 1) return OB_ERR_CUDA;
  int G = P->sms;  // one CTA per SM
  if (G > kGroupMax) G = kGroupMax;
  if ((rc = pool_reserve(P, 1, 0))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CallOrder co{P, s};
  if ((rc = co.begin())) return rc;
  if ((e = cudaMemsetAsync(P->gstate, 0, sizeof(GroupState), s)) != cudaSuccess) return cuda_fail(e);
  if ((e = launch_crr_group(G, s, (const obk::Opt*)params, (int)n_options, out, status, (double*)P->arena,
                            P->arena_bytes / sizeof(double), P->gstate, P->wide_wait_ns)) != cudaSuccess)
    return cuda_fail(e);
  return co.end();
}

int ob_greeks(const ob_option_t* params, int64_t n_options, double* out, double* grad, int32_t* status,
              void* stream) {
  if (n_options < 0 || n_options > (1 << 30)) return OB_ERR_ARG;
  if (n_options == 0) return OB_OK;
  if (!params || !out || !grad) return OB_ERR_ARG;
  const int n = (int)n_options;
  DevPool* P = nullptr;
  int dev = 0;
  int rc = pool_get(&P, &dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_call_mu[dev]);
  const int per_sm = 1;  // one CTA team per SM (8 or 16 warps, OB_GREEKS_WARPS)
  const int max_workers = P->sms * per_sm;
  const int workers = n < max_workers ? n : max_workers;
  if ((rc = pool_reserve(P, (size_t)n, (size_t)workers * (kGreeksSmBytes / per_sm)))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CallOrder co{P, s};
  if ((rc = co.begin())) return rc;
  cudaError_t e;
  if ((e = cudaMemsetAsync(P->ctl, 0, sizeof(int) * C_WORDS, s)) != cudaSuccess) return cuda_fail(e);
  const obk::Opt* opts = (const obk::Opt*)params;
  int* list0 = P->lists;
  int* list1 = P->lists + P->list_cap;
  size_t wbytes = P->arena_bytes / (size_t)workers;
  if (wbytes > kGreeksSmBytes / per_sm) wbytes = kGreeksSmBytes / per_sm;
  wbytes &= ~(size_t)255;
  e = P->greeks_warps == 16
          ? launch_greeks_team16(workers, s, opts, n, out, grad, status, P->arena, wbytes, P->ctl, list0,
                                 P->greeks_full)
          : launch_greeks_team8(workers, s, opts, n, out, grad, status, P->arena, wbytes, P->ctl, list0,
                                P->greeks_full);
  if (e != cudaSuccess) return cuda_fail(e);
  const size_t t1_bytes = (P->arena_bytes / kTier1Ctas) & ~(size_t)255;
  e = launch_greeks_retry(kTier1Ctas, s, opts, out, grad, status, P->arena, t1_bytes, &P->ctl[C_T0_OVF], list0,
                          &P->ctl[C_T1_HEAD], &P->ctl[C_T1_OVF], list1, 0);
  if (e != cudaSuccess) return cuda_fail(e);
  e = launch_greeks_retry(1, s, opts, out, grad, status, P->arena, P->arena_bytes & ~(size_t)255, &P->ctl[C_T1_OVF],
                          list1, &P->ctl[C_T2_HEAD], &P->ctl[C_T2_OVF], nullptr, 1);
  if (e != cudaSuccess) return cuda_fail(e);
  return co.end();
}

int ob_hedge_path(const ob_option_t* params, int64_t n_options, const int8_t* moves, int64_t stride,
                  double* out, double* hold, double* cash, int32_t* stop, int32_t* status, void* stream) {
  if (n_options < 0 || n_options > (1 << 30)) return OB_ERR_ARG;
  if (n_options == 0) return OB_OK;
  if (!params || !out || !hold || !stop || !moves || stride < 1 || stride > (1 << 26)) return OB_ERR_ARG;
  const int n = (int)n_options;
  DevPool* P = nullptr;
  int dev = 0;
  int rc = pool_get(&P, &dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_call_mu[dev]);
  const int workers = n < P->sms ? n : P->sms;  // one 16-warp CTA team per SM
  if ((rc = pool_reserve(P, (size_t)n, (size_t)workers * P->path_bytes))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CallOrder co{P, s};
  if ((rc = co.begin())) return rc;
  size_t wbytes = P->arena_bytes / (size_t)workers;
  if (wbytes > P->path_bytes) wbytes = P->path_bytes;
  wbytes &= ~(size_t)255;
  const obk::Opt* opts = (const obk::Opt*)params;
  cudaError_t e;
  if ((e = cudaMemsetAsync(P->ctl, 0, sizeof(int) * C_WORDS, s)) != cudaSuccess) return cuda_fail(e);
  const int* order = nullptr;  // the costliest options first, as in the batched form
  if (n <= kSortMax) {
    int npad = 1;
    while (npad < n) npad <<= 1;
    k_order<<<1, 1024, sizeof(unsigned long long) * npad, s>>>(opts, n, npad, P->order, P->ctl, workers * 16,
                                                                workers, 0.0);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    order = P->order;
  }
  // first tier: one slice per CTA; the options that outgrow it go to a second launch of one
  // CTA with the whole pool, where an option that still does not fit gets OB_ERR_CAPACITY
  int* list0 = P->lists;
  e = launch_path(workers, s, opts, n, nullptr, order, &P->ctl[C_HEAVY_HEAD], moves, (long long)stride, out, hold,
                  cash, stop, status, P->arena, wbytes, &P->ctl[C_T0_OVF], list0);
  if (e != cudaSuccess) return cuda_fail(e);
  e = launch_path(1, s, opts, n, &P->ctl[C_T0_OVF], list0, &P->ctl[C_T1_HEAD], moves, (long long)stride, out, hold,
                  cash, stop, status, P->arena, P->arena_bytes & ~(size_t)255, nullptr, nullptr);
  if (e != cudaSuccess) return cuda_fail(e);
  return co.end();
}

int ob_price_ask_bid_host(const ob_option_t* params, int64_t n_options, double* out,
                          int32_t* status) {
  if (n_options < 0 || n_options > (1 << 30)) return OB_ERR_ARG;
  if (n_options == 0) return OB_OK;
  if (!params || !out) return OB_ERR_ARG;
  DevPool* P = nullptr;
  int dev = 0;
  int rc = pool_get(&P, &dev);
  if (rc) return rc;
  cudaError_t e;
  // one host-buffer call at a time per device: the staging buffers are shared
  std::lock_guard<std::mutex> hl(g_host_mu[dev]);
  {
    if (!P->hstream) {
      if ((e = cudaStreamCreateWithFlags(&P->hstream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e);
    }
    if ((size_t)n_options > P->hcap) {
      cudaFree(P->hparams);
      cudaFree(P->hout);
      cudaFree(P->hstatus);
      P->hparams = nullptr; P->hout = nullptr; P->hstatus = nullptr; P->hcap = 0;
      if (cudaMalloc(&P->hparams, sizeof(ob_option_t) * n_options) != cudaSuccess ||
          cudaMalloc(&P->hout, sizeof(double) * 2 * n_options) != cudaSuccess ||
          cudaMalloc(&P->hstatus, sizeof(int) * n_options) != cudaSuccess) {
        cudaGetLastError();
        return OB_ERR_NOMEM;
      }
      P->hcap = (size_t)n_options;
    }
  }
  cudaStream_t s = P->hstream;
  if ((e = cudaMemcpyAsync(P->hparams, params, sizeof(ob_option_t) * n_options,
                           cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(e);
  rc = launch_tc(P->hparams, n_options, P->hout, P->hstatus, s, false);
  if (rc) return rc;
  if ((e = cudaMemcpyAsync(out, P->hout, sizeof(double) * 2 * n_options, cudaMemcpyDeviceToHost,
                           s)) != cudaSuccess)
    return cuda_fail(e);
  if (status && (e = cudaMemcpyAsync(status, P->hstatus, sizeof(int) * n_options,
                                     cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
  return OB_OK;
}

int ob_get_stats(ob_stats_t* host_out) {
  if (!host_out) return OB_ERR_ARG;
  DevPool* P = nullptr;
  int rc = pool_get(&P);
  if (rc) return rc;
  DevStats d;
  cudaError_t e = cudaMemcpy(&d, P->stats, sizeof(d), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e);
  host_out->options = (int64_t)d.options;
  host_out->node_updates = (int64_t)d.node_updates;
  host_out->u_points = (int64_t)d.upts;
  host_out->w_points = (int64_t)d.wpts;
  host_out->z_points = (int64_t)d.zpts;
  host_out->max_level_points = d.max_level;
  host_out->retried = d.retried;
  host_out->failed = d.failed;
  host_out->tiers = P->last_tiers;
  host_out->graph = P->last_graph;
  host_out->team_warps = P->team_warps;
  host_out->chip_points = (P->team_warps == 16 || P->team_warps == 8) ? chip_points(P, P->team_warps) : 0;
  host_out->half_teams = (P->team_warps == 16 && P->split_factor > 0.0 && host_out->chip_points == 0) ? 1 : 0;
  return OB_OK;
}

int ob_configure(int32_t team_warps, int32_t use_graphs, int32_t chip_points) {
  if (team_warps != 0 && team_warps != 4 && team_warps != 8 && team_warps != 12 && team_warps != 16)
    return OB_ERR_ARG;
  if (chip_points < -2) return OB_ERR_ARG;
  DevPool* P = nullptr;
  int dev = 0;
  int rc = pool_get(&P, &dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_call_mu[dev]);
  if (team_warps) P->team_warps = team_warps;
  if (use_graphs >= 0) P->use_graphs = use_graphs != 0;
  if (chip_points != -2) P->chip_req = chip_points;
  drop_graphs(P);
  return OB_OK;
}

int ob_autotune(const ob_option_t* params, int64_t n_options, int64_t sample, void* stream,
                int32_t* team_warps_out, int32_t* chip_out, float* ms_out) {
  if (n_options <= 0 || n_options > (1 << 30) || !params) return OB_ERR_ARG;
  const int n = (int)n_options;
  int m = (int)(sample > 0 && sample < n_options ? sample : n_options);
  const int stride = n / m;
  DevPool* P = nullptr;
  int dev = 0;
  int rc = pool_get(&P, &dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_call_mu[dev]);
  const int keep = P->team_warps;
  size_t need = 0;
  for (int tw : {16, 12, 8, 4}) {
    P->team_warps = tw;
    const size_t b = batched_need(P, m);
    if (b > need) need = b;
  }
  P->team_warps = keep;
  if ((rc = pool_reserve(P, (size_t)m, need))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CallOrder co{P, s};
  if ((rc = co.begin())) return rc;
  cudaError_t e;
  if (m > P->tune_cap) {
    cudaFree(P->tune_params);
    cudaFree(P->tune_out);
    cudaFree(P->tune_status);
    P->tune_params = nullptr; P->tune_out = nullptr; P->tune_status = nullptr; P->tune_cap = 0;
    if (cudaMalloc(&P->tune_params, sizeof(obk::Opt) * m) != cudaSuccess ||
        cudaMalloc(&P->tune_out, sizeof(double) * 2 * m) != cudaSuccess ||
        cudaMalloc(&P->tune_status, sizeof(int) * m) != cudaSuccess) {
      cudaGetLastError();
      return OB_ERR_NOMEM;
    }
    P->tune_cap = m;
  }
  k_gather<<<(m + 255) / 256, 256, 0, s>>>((const obk::Opt*)params, n, stride, m, P->tune_params);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
  cudaEvent_t a = nullptr, b = nullptr;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return cuda_fail(e);
  }
  // candidates: team width, on-chip w points per CTA (0: w in the global scratch; -1: the
  // fused level step with all the shared memory a CTA can take), and whether 16-warp CTAs
  // split into two 8-warp teams for the light options
  const int cands[kTuneCands][3] = {{16, 0, 1}, {16, 0, 0}, {12, 0, 0}, {8, 0, 0}, {4, 0, 0}, {16, -1, 0}, {8, -1, 0}};
  const int keep_chip = P->chip_req;
  const double keep_split = P->split_factor;
  const double split_on = keep_split > 0.0 ? keep_split : kSplitFactor;
  int best = keep, best_chip = keep_chip;
  double best_split = keep_split;
  float best_ms = 0.0f;
  for (int c = 0; c < kTuneCands && rc == OB_OK; ++c) {
    P->team_warps = cands[c][0];
    P->chip_req = cands[c][1];
    P->split_factor = cands[c][2] ? split_on : 0.0;
    float ms = 0.0f;
    for (int rep = 0; rep < 2 && rc == OB_OK; ++rep) {  // one warm-up run, one timed run
      if ((e = cudaEventRecord(a, s)) != cudaSuccess) { rc = cuda_fail(e); break; }
      rc = enqueue_batched(P, P->tune_params, m, P->tune_out, P->tune_status, s);
      if (rc) break;
      if ((e = cudaEventRecord(b, s)) != cudaSuccess || (e = cudaEventSynchronize(b)) != cudaSuccess ||
          (e = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) {
        rc = cuda_fail(e);
        break;
      }
    }
    if (rc) break;
    if (ms_out) ms_out[c] = ms;
    // a later candidate must beat the best so far by 1 %: the sample's timings are close for
    // the first two, and a timing's noise should not move the choice
    if (c == 0 || ms < 0.99f * best_ms) {
      best_ms = ms;
      best = cands[c][0];
      best_chip = cands[c][1];
      best_split = P->split_factor;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  P->team_warps = rc ? keep : best;
  P->chip_req = rc ? keep_chip : best_chip;
  P->split_factor = rc ? keep_split : best_split;
  drop_graphs(P);
  if (team_warps_out) *team_warps_out = P->team_warps;
  if (chip_out) *chip_out = chip_points(P, P->team_warps);
  if (rc) return rc;
  return co.end();
}

int ob_release(void) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  std::lock_guard<std::mutex> hl(g_host_mu[dev]);
  std::lock_guard<std::mutex> cl(g_call_mu[dev]);
  std::lock_guard<std::mutex> lk(g_mu);
  DevPool& P = g_pool[dev];
  if (!P.init) return OB_OK;
  cudaDeviceSynchronize();
  drop_graphs(&P);
  if (P.order_ev) cudaEventDestroy(P.order_ev);
  if (P.cap_stream) cudaStreamDestroy(P.cap_stream);
  cudaFree(P.gstate);
  cudaFree(P.tune_params);
  cudaFree(P.tune_out);
  cudaFree(P.tune_status);
  cudaFree(P.arena);
  cudaFree(P.ctl);
  cudaFree(P.order);
  cudaFree(P.lists);
  cudaFree(P.stats);
  cudaFree(P.hparams);
  cudaFree(P.hout);
  cudaFree(P.hstatus);
  if (P.hstream) cudaStreamDestroy(P.hstream);
  P = DevPool();
  return OB_OK;
}

const char* ob_strerror(int code) {
  switch (code) {
    case OB_OK: return "ok";
    case OB_ERR_ARG: return "invalid argument or option parameter";
    case OB_ERR_ARBITRAGE: return "tree admits arbitrage (d < r < u fails)";
    case OB_ERR_CAPACITY: return "piecewise-linear functions outgrew the scratch pool";
    case OB_ERR_TIMEOUT: return "bounded device wait expired";
    case OB_ERR_CUDA: return "CUDA runtime error";
    case OB_ERR_NOMEM: return "scratch pool allocation failed";
    default: return "unknown status code";
  }
}

const char* ob_last_cuda_error(void) { return g_cuda_err; }

int ob_fp64_peak(int64_t iters, void* stream, double* tflops_out, double* ms_out) {
  if (iters <= 0 || !tflops_out) return OB_ERR_ARG;
  DevPool* P = nullptr;
  int dev = 0;
  int rc = pool_get(&P, &dev);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_call_mu[dev]);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  const int blocks = P->sms * 8, threads = 256;  // 64 warps per SM
  cudaEvent_t a = nullptr, b = nullptr;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return cuda_fail(e);
  }
  float best = 0.0f;
  for (int rep = 0; rep < 3 && rc == OB_OK; ++rep) {  // the first run warms the clocks
    float ms = 0.0f;
    if ((e = cudaEventRecord(a, s)) != cudaSuccess) { rc = cuda_fail(e); break; }
    k_fp64_probe<<<blocks, threads, 0, s>>>((long long)iters, 0.999999999, 1e-9, (double*)P->ctl);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventRecord(b, s)) != cudaSuccess ||
        (e = cudaEventSynchronize(b)) != cudaSuccess || (e = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) {
      rc = cuda_fail(e);
      break;
    }
    if (rep == 1 || (rep > 1 && ms < best)) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  const double flops = 2.0 * kProbeChains * (double)iters * blocks * threads;
  *tflops_out = flops / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return OB_OK;
}

int ob_price_ask_bid_noalloc(const ob_option_t* params, int64_t n_options, double* out,
                             int32_t* status, void* stream) {
  if (n_options < 0 || n_options > kNoAllocMaxOptions) return OB_ERR_ARG;
  if (n_options == 0) return OB_OK;
  if (!params || !out) return OB_ERR_ARG;
  const int n = (int)n_options;
  char* base = nullptr;
  int rc = noalloc_base(&base);
  if (rc) return rc;
  cudaError_t e;
  int* ctl = (int*)base;
  DevStats* ds = (DevStats*)(base + 256);
  int* order = (int*)(base + kNoAllocHead);
  int* list0 = (int*)(base + kNoAllocHead + sizeof(int) * (size_t)kNoAllocMaxOptions);
  int* list1 = list0 + kNoAllocMaxOptions;
  char* arena = base + kNoAllocHead + sizeof(int) * (size_t)kNoAllocMaxOptions + kNoAllocLists;
  const size_t arena_bytes = (kNoAllocBytes - (size_t)(arena - base)) & ~(size_t)255;
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: reset the queues and counters
  if ((e = cudaMemsetAsync(base, 0, kNoAllocHead, s)) != cudaSuccess) return cuda_fail(e);
  const obk::Opt* opts = (const obk::Opt*)params;
  int npad = 1;
  while (npad < n) npad <<= 1;
  k_order<<<1, 1024, sizeof(unsigned long long) * npad, s>>>(opts, n, npad, order, ctl,
                                                             kNoAllocCtas * kNW, kNoAllocCtas,
                                                             kHeavyFactor);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
  const size_t cta_bytes = (arena_bytes / kNoAllocCtas) & ~(size_t)255;
  // every option goes to a CTA team (heavy factor 0), as in the pooled form
  {
    const BatchedArgs ba{opts, n, order, out, status, arena, cta_bytes, ctl, list0, ds, 0, nullptr};
    if ((e = launch_batched_narrow(kNW, false, false, kNoAllocCtas, 0, s, ba)) != cudaSuccess) return cuda_fail(e);
  }
  if ((e = launch_retry(1, s, opts, out, status, arena, arena_bytes, &ctl[C_T0_OVF], list0, &ctl[C_T1_HEAD],
                        &ctl[C_T1_OVF], list1, 1, ds, nullptr)) != cudaSuccess)
    return cuda_fail(e);
  return OB_OK;
}


}  // extern "C"
