// ob_kern.cuh -- what the library's translation units share: constants, the
// per-call counters, option checks, the per-option drivers of the kernels, the
// batched and Greeks team kernels (templates, instantiated in the units that launch
// them) and the launch functions each unit defines for the host code in ob_lib.cu.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ob.h"
#include "ob_adj.cuh"
#include "ob_tc.cuh"

namespace obl {

constexpr int kBlock = 128;          // CTA of the plain kernel and of the CRR kernel (4 warps)
constexpr int kNW = 8;               // warps of a CTA of the batched kernel
constexpr int kTeamBlock = 32 * kNW;
constexpr int kTiers = 3;            // launches per ob_price_ask_bid call
constexpr int kTier1Ctas = 16;       // CTAs of the first follow-up launch
constexpr int kSortMax = 8192;       // largest batch ordered by cost
constexpr int kCrrSmem = 2304;       // doubles of shared memory per CRR warp (N <= 2303)
constexpr double kHeavyFactor = 0.0; // heavy: predicted cost > factor x (total / warps); 0: all
constexpr double kSplitFactor = 0.04; // 16-warp CTAs: half-CTA teams below factor x (total / CTAs)
// control words
enum { C_HEAVY_HEAD = 0, C_LIGHT_HEAD = 1, C_NHEAVY = 2, C_T0_OVF = 3, C_T1_HEAD = 4, C_T1_OVF = 5,
       C_T2_HEAD = 6, C_T2_OVF = 7, C_WORDS = 8 };

constexpr int ST_TIMEOUT = -4;  // OB_ERR_TIMEOUT: a bounded device wait ran out

struct DevStats {
  unsigned long long options, node_updates, upts, wpts, zpts;
  int max_level, retried, failed, tiers;
};

static_assert(sizeof(ob_option_t) == 64, "ob_option_t must be 64 bytes");
static_assert(sizeof(obk::Opt) == 64, "Opt must be 64 bytes");

__device__ __forceinline__ double dnan() { return __longlong_as_double(0x7ff8000000000000LL); }

__device__ __forceinline__ int check_option(const obk::Opt& o, bool need_k) {
  if (!(o.N >= 1) || o.N > (1 << 26) || !(o.S0 > 0.0) || !(o.sigma > 0.0) || !(o.T > 0.0) ||
      !(o.K >= 0.0) || !isfinite(o.R) || !isfinite(o.S0) || !isfinite(o.K) || !isfinite(o.sigma) ||
      !isfinite(o.T) || o.payoff < 0 || o.payoff > 2)
    return obk::ST_ARG;
  if (need_k && !(o.k >= 0.0 && o.k < 1.0)) return obk::ST_ARG;
  if (o.payoff == obk::PAY_SPREAD && !(o.K2 >= o.K && isfinite(o.K2))) return obk::ST_ARG;
  return obk::ST_OK;
}

// ------------------------------------------------------------------ ordering
// Predicted work of an option: node updates times an estimate of the
// breakpoints per node (both parties).  Puts keep about one breakpoint per
// node and party; calls and cash-settled spreads gather many once
// x = k / (sigma sqrt(T/N)) exceeds ~1 (pieces whose slopes stay inside the
// bid/ask window survive more levels).  Fitted to the oracle's counts on the
// batched workload; only the ordering and the warp/CTA split depend on it.
__device__ __forceinline__ double predicted_cost(const obk::Opt& o) {
  const double N = o.N > 0 ? (double)o.N : 1.0;
  const double nodes = (N + 1.0) * (N + 2.0) * 0.5;
  const double sd = (o.sigma > 0.0 && o.T > 0.0) ? o.sigma * sqrt(o.T / N) : 1.0;
  const double x = (o.k > 0.0) ? o.k / sd : 0.0;
  double m = 2.0;
  if (x > 1.0) {
    if (o.payoff == obk::PAY_CALL) m += 1.5 * x;
    else if (o.payoff == obk::PAY_SPREAD) m += x * x;
  }
  double c = nodes * m;
  return c < 1e12 ? c : 1e12;
}

// ------------------------------------------------------------------ induction with costs
template <class Team, bool CHIP = false>
__device__ __forceinline__ void price_one(const Team& tm, const obk::Opt& o, char* slice, size_t bytes,
                                          int& rc, double& ask, double& bid, obk::Stats& st,
                                          const obk::WBuf* chip = nullptr) {
  rc = check_option(o, true);
  ask = dnan();
  bid = dnan();
  st.upts = st.wpts = st.zpts = 0;
  st.zmax_level = 0;
  for (int c = 0; c < 4; ++c) st.hedge[c] = dnan();
  if (rc != obk::ST_OK) return;
  obk::Lay L;
  if (!obk::carve(slice, bytes, o.N, 2 * (o.N + 2), L)) {
    rc = obk::ST_CAPACITY;
    return;
  }
  obk::TcRun<Team, CHIP> R(tm, o, L);
  if (CHIP) R.chip = *chip;
  rc = R.run(ask, bid);
  st = R.st;
}

// Record an option's result (one thread); a capacity failure goes to the retry
// list when a follow-up launch exists.
__device__ __forceinline__ void finish(int oi, int rc, double ask, double bid, const obk::Stats& st,
                                       const obk::Opt& o, double* out, int* status, int* ovf_count,
                                       int* ovf_list, bool retry, DevStats* ds, double* hedge) {
  if (rc == obk::ST_CAPACITY && retry) {
    const int pos = atomicAdd(ovf_count, 1);
    ovf_list[pos] = oi;
    atomicAdd(&ds->retried, 1);
    return;
  }
  out[2 * oi] = rc ? dnan() : ask;
  out[2 * oi + 1] = rc ? dnan() : bid;
  if (hedge)
    for (int c = 0; c < 4; ++c) hedge[4 * (size_t)oi + c] = rc ? dnan() : st.hedge[c];
  if (status) status[oi] = rc;
  atomicAdd(&ds->options, 1ULL);
  if (rc == obk::ST_OK) {
    const unsigned long long N = (unsigned long long)o.N;
    atomicAdd(&ds->node_updates, (N + 1) * (N + 2) / 2);
    atomicAdd(&ds->upts, (unsigned long long)st.upts);
    atomicAdd(&ds->wpts, (unsigned long long)st.wpts);
    atomicAdd(&ds->zpts, (unsigned long long)st.zpts);
    atomicMax(&ds->max_level, st.zmax_level);
  } else {
    atomicAdd(&ds->failed, 1);
  }
}

// Batched form.  Every CTA first takes the costliest options (order[0..nheavy))
// one at a time as a whole-CTA team, then the remaining options one at a time from a
// second queue: each of its warps (WARPS), or each half of the CTA as a team of NW/2 warps
// with its own barrier (HALVES), so that two options share the SM and one team's waits
// at its barriers overlap the other's work.  Both queues are device counters.
// CHIP: the CTA's dynamic shared memory holds the w arrays of chip_points points (the
// fused level step of CTA teams, TcRun::level_fused).
template <int NW>
struct BatchedTbuf {  // exchange area of the CTA team, or of its two halves
  static constexpr int whole = obk::BlockTeam<NW>::BUF, halves = 2 * obk::BlockTeam<NW / 2, true>::BUF;
  static constexpr int value = whole > halves ? whole : halves;
};

// The second phase of the HALVES form: the CTA as two teams of NW/2 warps, each with its
// own barrier and half the CTA's scratch, taking options from the light queue.  Not
// inlined: the kernel's first phase keeps its own register allocation.
template <int NW>
__device__ __noinline__ void batched_halves(const obk::Opt* __restrict__ opts, int n,
                                            const int* __restrict__ order, double* out, int* status,
                                            char* my, size_t cta_bytes, int* ctl, int* ovf_list,
                                            DevStats* ds, double* hedge, long long* tbuf, int nh) {
  constexpr int HW = NW / 2;
  using Half = obk::BlockTeam<HW, true>;
  const int h = threadIdx.x >= 32 * HW ? 1 : 0;
  const Half ht{tbuf + h * Half::BUF, 32 * HW * h, 1 + h};
  const size_t hbytes = (cta_bytes / 2) & ~(size_t)255;
  char* hmy = my + (size_t)h * hbytes;
  for (;;) {
    int v = 0;
    if (ht.lane() == 0) v = atomicAdd(&ctl[C_LIGHT_HEAD], 1);
    const int idx = ht.bcast0(v) + nh;
    if (idx >= n) break;
    const int oi = order[idx];
    const obk::Opt o = opts[oi];
    int rc;
    double ask, bid;
    obk::Stats st;
    price_one(ht, o, hmy, hbytes, rc, ask, bid, st);
    if (ht.lane() == 0) finish(oi, rc, ask, bid, st, o, out, status, &ctl[C_T0_OVF], ovf_list, true, ds, hedge);
    ht.sync();
  }
}

template <int NW, bool WARPS, bool CHIP = false, bool HALVES = false>
__global__ void __launch_bounds__(32 * NW, 16 / NW) k_tc_batched(
    const obk::Opt* __restrict__ opts, int n, const int* __restrict__ order, double* out, int* status,
    char* arena, size_t cta_bytes, int* ctl, int* ovf_list, DevStats* ds, int chip_points, double* hedge) {
  static_assert(!(HALVES && (WARPS || CHIP || NW % 2)), "HALVES: even NW, no warp tail, no chip");
  __shared__ long long tbuf[HALVES ? BatchedTbuf<NW>::value : obk::BlockTeam<NW>::BUF];
  extern __shared__ __align__(16) char chip_smem[];
  obk::BlockTeam<NW> bt{tbuf};
  const obk::WBuf chip = obk::carve_wbuf(chip_smem, chip_points);
  char* my = arena + (size_t)blockIdx.x * cta_bytes;
  const int nh = order ? *((volatile int*)&ctl[C_NHEAVY]) : 0;
  for (;;) {
    int v = 0;
    if (threadIdx.x == 0) v = atomicAdd(&ctl[C_HEAVY_HEAD], 1);
    const int idx = bt.bcast0(v);
    if (idx >= nh) break;
    const int oi = order[idx];
    const obk::Opt o = opts[oi];
    int rc;
    double ask, bid;
    obk::Stats st;
    price_one<obk::BlockTeam<NW>, CHIP>(bt, o, my, cta_bytes, rc, ask, bid, st, &chip);
    if (threadIdx.x == 0) finish(oi, rc, ask, bid, st, o, out, status, &ctl[C_T0_OVF], ovf_list, true, ds, hedge);
    bt.sync();
  }
  if (HALVES) {
    __syncthreads();  // the whole-CTA team's last exchange is read before tbuf is reused
    batched_halves<NW>(opts, n, order, out, status, my, cta_bytes, ctl, ovf_list, ds, hedge, tbuf, nh);
    return;
  }
  if (!WARPS) return;  // every option went to a CTA team
  obk::WarpTeam wt;
  const size_t wbytes = (cta_bytes / NW) & ~(size_t)255;
  char* wmy = my + (size_t)(threadIdx.x >> 5) * wbytes;
  for (;;) {
    int v = 0;
    if (wt.lane() == 0) v = atomicAdd(&ctl[C_LIGHT_HEAD], 1);
    const int idx = wt.bcast0(v) + nh;
    if (idx >= n) break;
    const int oi = order ? order[idx] : idx;
    const obk::Opt o = opts[oi];
    int rc;
    double ask, bid;
    obk::Stats st;
    price_one(wt, o, wmy, wbytes, rc, ask, bid, st);
    if (wt.lane() == 0) finish(oi, rc, ask, bid, st, o, out, status, &ctl[C_T0_OVF], ovf_list, true, ds, hedge);
    wt.sync();
  }
}

// ------------------------------------------------------------------ whole-GPU form
// Each option in turn on every SM: the CTAs split each level's nodes (TcGroup) and
// meet at two grid barriers per level.  Launched cooperatively, so all CTAs are
// resident; every wait is bounded.
constexpr int kGroupMax = 1024;                                    // CTAs of the grid at most
constexpr unsigned long long kGroupWaitNs = 10000000000ULL;        // 10 s per barrier wait
constexpr int kGroupNW = 16;                                       // warps per CTA
constexpr int kTrapD = 8;         // levels of a trapezoid round of the whole-GPU form
constexpr int kTrapPoints = 128;  // a level is light below this many points per CTA
constexpr int kTrapColumnPoints = 8;  // ... and this many per column on average (small nodes)
constexpr double kWideSplitX = 6.0;   // nodes split over CTAs when k > this x sigma sqrt(dt)
constexpr int kSplitExtraPoints = 4000;  // ... on levels whose largest node exceeds a share by this

struct GroupState {
  unsigned int count;  // arrivals at the current barrier
  unsigned int gen;    // barriers completed
  int err;             // a wait ran out: every later barrier fails at once
  int pad;
  int cnt[2][kGroupMax];  // points of each CTA's share of a level (-1: overflow)
  obk::SplitRec sr[kGroupMax];  // each CTA's share of a level whose nodes are split (TcSplit)
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ------------------------------------------------------------------ adjoint (Greeks)
template <class Team>
__device__ __forceinline__ void greeks_one(const Team& tm, const obk::Opt& o, char* slice, size_t bytes,
                                           int& rc, double& ask, double& bid, double* gA, double* gB,
                                           bool allow_full = true) {
  rc = check_option(o, true);
  ask = dnan();
  bid = dnan();
  if (rc != obk::ST_OK) return;
  obk::Lay L;
  obk::AdjLay A;
  // full mode (records of every level, no recompute) when the predicted records fit:
  // 2 doubles and about 2.5 ints per point of w, taken as twice the predicted breakpoints.
  // A misprediction ends in ST_CAPACITY, and the follow-up launches (allow_full false:
  // checkpoints, larger slices) price the option.
  const double wpred = 2.0 * predicted_cost(o);
  const bool full = allow_full && obk::carve_greeks(slice, bytes, o.N, 2 * (o.N + 2), L, A, true) &&
                    2.0 * wpred < (double)A.rd_cap && 2.5 * wpred < (double)A.ri_cap;
  if (!full && !obk::carve_greeks(slice, bytes, o.N, 2 * (o.N + 2), L, A, false)) {
    rc = obk::ST_CAPACITY;
    return;
  }
  obk::TcRun<Team> R(tm, o, L);
  obk::TcAdj<Team> G(R, A);
  rc = G.run(ask, bid, gA, gB, full);
}

__device__ __forceinline__ void greeks_finish(int oi, int rc, double ask, double bid, const double* gA,
                                              const double* gB, double* out, double* grad, int* status,
                                              int* ovf_count, int* ovf_list, bool retry) {
  if (rc == obk::ST_CAPACITY && retry) {
    const int pos = atomicAdd(ovf_count, 1);
    ovf_list[pos] = oi;
    return;
  }
  out[2 * oi] = rc ? dnan() : ask;
  out[2 * oi + 1] = rc ? dnan() : bid;
  for (int k = 0; k < obk::NPAR; ++k) {
    grad[12 * (size_t)oi + k] = rc ? dnan() : gA[k];
    grad[12 * (size_t)oi + 6 + k] = rc ? dnan() : gB[k];
  }
  if (status) status[oi] = rc;
}

// Greeks on CTA teams: each CTA takes options from the queue over [0, n) as one team.
template <int NW>
__global__ void __launch_bounds__(32 * NW, NW >= 16 ? 1 : 8 / NW) k_greeks_team(
    const obk::Opt* __restrict__ opts, int n, double* out, double* grad, int* status, char* arena,
    size_t cta_bytes, int* ctl, int* ovf_list, int allow_full) {
  __shared__ long long tbuf[obk::BlockTeam<NW>::BUF];
  obk::BlockTeam<NW> bt{tbuf};
  char* my = arena + (size_t)blockIdx.x * cta_bytes;
  for (;;) {
    int v = 0;
    if (threadIdx.x == 0) v = atomicAdd(&ctl[C_LIGHT_HEAD], 1);
    const int oi = bt.bcast0(v);
    if (oi >= n) break;
    const obk::Opt o = opts[oi];
    int rc;
    double ask, bid, gA[obk::NPAR], gB[obk::NPAR];
    greeks_one(bt, o, my, cta_bytes, rc, ask, bid, gA, gB, allow_full != 0);
    if (threadIdx.x == 0) greeks_finish(oi, rc, ask, bid, gA, gB, out, grad, status, &ctl[C_T0_OVF], ovf_list, true);
    bt.sync();
  }
}


// ------------------------------------------------------------------ plain CRR (no costs)
// c_{t,j} = max(P_{t,j}, pu c_{t+1,j+1} + pd c_{t+1,j}), pu = p/r, pd = (1-p)/r, with the
// exercise value P = max(payoff, 0) tabulated per option by stock exponent 2j - t.
__device__ __forceinline__ double crr_payoff(const obk::Opt& o, double S) {
  double v;
  if (o.payoff == obk::PAY_PUT) v = o.K - S;
  else if (o.payoff == obk::PAY_CALL) v = S - o.K;
  else v = fmax(S - o.K, 0.0) - fmax(S - o.K2, 0.0);
  return fmax(v, 0.0);
}

// One node update; both CRR kernels use it, so their results agree bit for bit.  The
// values are >= 0, so their bit patterns order like the values.
__device__ __forceinline__ double crr_step(double pu, double pd, double up, double cur, double ex) {
  const double cont = fma(pu, up, pd * cur);
  return (__double_as_longlong(cont) > __double_as_longlong(ex)) ? cont : ex;
}

// ------------------------------------------------------------------ launch functions
// Arguments of the batched kernel.
struct BatchedArgs {
  const obk::Opt* opts;
  int n;
  const int* order;
  double* out;
  int* status;
  char* arena;
  size_t cta_bytes;
  int* ctl;
  int* ovf_list;
  DevStats* ds;
  int chip_points;
  double* hedge;  // may be null: the hedge at the root, 4 doubles per option
};

// k_tc_batched<nw, warps, chip> on `grid` CTAs (ob_batched16.cu: nw 16, 12; ob_batched8.cu:
// nw 8, 4 and the on-chip instantiations of nw 16, 8).
cudaError_t launch_batched_wide(int nw, bool warps, int grid, cudaStream_t s, const BatchedArgs& a);
// ob_batched_half.cu
cudaError_t launch_batched_halves(int grid, cudaStream_t s, const BatchedArgs& a);
cudaError_t launch_batched_narrow(int nw, bool warps, bool chip, int grid, size_t smem, cudaStream_t s,
                                  const BatchedArgs& a);
cudaError_t set_chip_smem(int bytes16, int bytes8);

// ob_tiers.cu
cudaError_t launch_retry(int grid, cudaStream_t s, const obk::Opt* opts, double* out, int* status, char* arena,
                         size_t cta_bytes, const int* in_count, const int* in_list, int* head, int* ovf_count,
                         int* ovf_list, int last, DevStats* ds, double* hedge);
cudaError_t launch_plain(int blocks, cudaStream_t s, const obk::Opt* opts, int n, double* out, int* status,
                         char* arena, size_t wbytes, int nworkers, DevStats* ds);

// ob_group.cu
cudaError_t group_occupancy(int* per_sm);
cudaError_t crr_group_occupancy(int* per_sm);
cudaError_t launch_crr_group(int G, cudaStream_t s, const obk::Opt* opts, int n, double* out, int* status,
                             double* buf, size_t buf_doubles, GroupState* gs, unsigned long long wait_ns);
cudaError_t launch_group(int G, cudaStream_t s, const obk::Opt* opts, int n, double* out, int* status,
                         char* arena, size_t shared_bytes, size_t cta_bytes, GroupState* gs, DevStats* ds,
                         unsigned long long wait_ns, int skip_cta, double split_x);

// ob_greeks8.cu (8- and 16-warp CTA teams) and ob_greeks.cu (the follow-up launches)
cudaError_t launch_greeks_team8(int grid, cudaStream_t s, const obk::Opt* opts, int n, double* out, double* grad,
                                int* status, char* arena, size_t cta_bytes, int* ctl, int* ovf_list, int allow_full);
cudaError_t launch_greeks_team16(int grid, cudaStream_t s, const obk::Opt* opts, int n, double* out, double* grad,
                                 int* status, char* arena, size_t cta_bytes, int* ctl, int* ovf_list, int allow_full);
cudaError_t launch_greeks_retry(int grid, cudaStream_t s, const obk::Opt* opts, double* out, double* grad,
                                int* status, char* arena, size_t cta_bytes, const int* in_count,
                                const int* in_list, int* head, int* ovf_count, int* ovf_list, int last);

// ob_path.cu (the hedge along a path: one 16-warp CTA team per option from a device queue)
cudaError_t launch_path(int grid, cudaStream_t s, const obk::Opt* opts, int n, const int* n_dev, const int* order,
                        int* head, const int8_t* moves, long long stride, double* out, double* hold, double* cash,
                        int* stop, int* status, char* arena, size_t cta_bytes, int* ovf_count, int* ovf_list);

}  // namespace obl
