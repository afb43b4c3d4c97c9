// ob_group.cu -- the whole-GPU forms: one cooperative launch of a CTA per SM, each
// option in turn with every level split over all CTAs (TcGroup for the induction with
// costs, trapezoid tiles of levels for the plain CRR recursion), bounded grid barriers.
#include "ob_kern.cuh"

namespace obl {

// Barrier of all CTAs of the grid.  Thread 0 publishes with a fence and an atomic
// arrival, the last arrival releases the others by bumping the generation; a wait
// longer than wait_ns (or 2^30 polls) sets err.  Returns false once err is set.
__device__ bool grid_barrier(GroupState* gs, unsigned& gen, unsigned long long wait_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = *((volatile int*)&gs->err) == 0;
    if (ok) {
      const unsigned want = gen + 1u;
      __threadfence();
      const unsigned arrived = atomicAdd(&gs->count, 1u) + 1u;
      if (arrived == gridDim.x) {
        atomicExch(&gs->count, 0u);
        __threadfence();
        atomicExch(&gs->gen, want);
      } else {
        const unsigned long long t0 = global_ns();
        for (unsigned it = 0;; ++it) {
          if (*((volatile unsigned*)&gs->gen) == want) break;
          if (*((volatile int*)&gs->err) != 0) { ok = 0; break; }
          if (it > (1u << 30) || global_ns() - t0 > wait_ns) {
            atomicExch(&gs->err, 1);
            ok = 0;
            break;
          }
          __nanosleep(128);
        }
      }
      __threadfence();
      gen = want;
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// One level t of k_tc_group with its nodes split over the CTAs (TcSplit): pass 1 and the
// share's pass 2, a grid barrier; the running minima across shares and the boundary points,
// a barrier; pass 3, a barrier for the counts; the copy into the shared level, a barrier.
// Returns the status every CTA agrees on.
__device__ __forceinline__ int split_level(obk::TcSplit<obk::BlockTeam<kGroupNW>>& sp, int t, int G, int c,
                                           GroupState* gs, unsigned& gen, unsigned long long wait_ns,
                                           int* s_cnt, obk::Stats& acc) {
  const obk::Stats before = sp.R.st;
  sp.phase_a(t, gs->sr);
  if (!grid_barrier(gs, gen, wait_ns)) return ST_TIMEOUT;
  if (obk::TcSplit<obk::BlockTeam<kGroupNW>>::overflow(gs->sr, G)) return obk::ST_CAPACITY;
  sp.phase_b(gs->sr);
  if (!grid_barrier(gs, gen, wait_ns)) return ST_TIMEOUT;
  const bool ok = sp.phase_c(t, gs->sr);
  acc.upts += sp.R.st.upts - before.upts;
  acc.wpts += sp.R.st.wpts - before.wpts;
  acc.zpts += sp.R.st.zpts - before.zpts;
  if (threadIdx.x == 0) gs->cnt[t & 1][c] = ok ? sp.ztot : -1;
  if (!grid_barrier(gs, gen, wait_ns)) return ST_TIMEOUT;
  int bad = 0;
  for (int k = threadIdx.x; k < G; k += blockDim.x) {
    s_cnt[k] = __ldcg(&gs->cnt[t & 1][k]);
    if (s_cnt[k] < 0) bad = 1;
  }
  if (__syncthreads_or(bad)) return obk::ST_CAPACITY;
  if (!sp.publish(t, s_cnt)) return obk::ST_CAPACITY;
  if (sp.R.st.zmax_level > acc.zmax_level) acc.zmax_level = sp.R.st.zmax_level;
  if (!grid_barrier(gs, gen, wait_ns)) return ST_TIMEOUT;
  return obk::ST_OK;
}

// One trapezoid round of k_tc_group from the complete shared level B (TcTrap): this CTA's
// window of columns down D levels, the grid barrier for the counts, the copy into the shared
// level B - D and the barrier that ends the round.  Sets t to the next level to compute
// (B - D - 1) and returns the status every CTA agrees on.
__device__ __forceinline__ int trap_round(obk::TcTrap<obk::BlockTeam<kGroupNW>>& tr, int B, int G, int c,
                                          GroupState* gs, unsigned& gen, unsigned long long wait_ns,
                                          int* s_cnt, int* s_cnt2, obk::Stats& acc, int& t) {
  int D, Ga, a, b;
  tr.plan(B, kTrapD, G, c, D, Ga, a, b);
  const obk::Stats before = tr.R.st;
  const bool ok = tr.compute(B, D, a, b);
  acc.upts += tr.R.st.upts - before.upts;
  acc.wpts += tr.R.st.wpts - before.wpts;
  acc.zpts += tr.R.st.zpts - before.zpts;
  if (threadIdx.x == 0) {
    gs->cnt[0][c] = ok ? tr.nS : -1;
    gs->cnt[1][c] = ok ? tr.nB : 0;
  }
  if (!grid_barrier(gs, gen, wait_ns)) return ST_TIMEOUT;
  int bad = 0;
  for (int k = threadIdx.x; k < G; k += blockDim.x) {
    s_cnt[k] = __ldcg(&gs->cnt[0][k]);
    s_cnt2[k] = __ldcg(&gs->cnt[1][k]);
    if (s_cnt[k] < 0) bad = 1;
  }
  if (__syncthreads_or(bad)) return obk::ST_CAPACITY;
  if (!tr.publish(B - D, G, c, s_cnt, s_cnt2)) return obk::ST_CAPACITY;
  if (tr.R.st.zmax_level > acc.zmax_level) acc.zmax_level = tr.R.st.zmax_level;
  if (!grid_barrier(gs, gen, wait_ns)) return ST_TIMEOUT;
  t = B - D - 1;
  return obk::ST_OK;
}

// How an option runs on the whole GPU.  Trapezoid rounds (1) where the columns carry about
// the same work: puts, and calls whose cost rate stays below one step's move (spreads gather
// breakpoints around their strikes, and a round's halo columns would repeat that work).
// Nodes split over the CTAs (2) where large nodes would leave most CTAs waiting: calls and
// spreads with k > split_x sigma sqrt(dt), on the levels whose largest node outgrows a share
// (split_x < 0: every level of every such option, a test control).  Otherwise shares of
// whole nodes (0).
enum { WIDE_NODES = 0, WIDE_TRAP = 1, WIDE_SPLIT = 2 };
__device__ __forceinline__ int wide_mode(const obk::Opt& o, double split_x) {
  if (o.payoff == obk::PAY_PUT) return WIDE_TRAP;
  if (!(o.N >= 1) || !(o.sigma > 0.0) || !(o.T > 0.0) || !(o.k >= 0.0)) return WIDE_NODES;
  const double step = o.sigma * sqrt(o.T / o.N);
  if (o.payoff == obk::PAY_CALL && o.k <= step) return WIDE_TRAP;
  return (o.k > split_x * step) ? WIDE_SPLIT : WIDE_NODES;
}

// MODE: the options of that wide_mode; the three instantiations run one after the other on
// the call's stream, so each keeps its own register allocation.
template <int MODE>
__global__ void __launch_bounds__(32 * kGroupNW, 1) k_tc_group(
    const obk::Opt* __restrict__ opts, int n, double* out, int* status, char* arena,
    size_t shared_bytes, size_t cta_bytes, GroupState* gs, DevStats* ds, unsigned long long wait_ns,
    int skip_cta, double split_x) {
  __shared__ long long tbuf[obk::BlockTeam<kGroupNW>::BUF];
  __shared__ int s_cnt[kGroupMax], s_cnt2[kGroupMax], s_max;
  obk::BlockTeam<kGroupNW> bt{tbuf};
  const int G = gridDim.x, c = blockIdx.x;
  // test control: this CTA never arrives at any barrier, so the others' bounded waits
  // run out and every option of the call reports OB_ERR_TIMEOUT
  if (c == skip_cta) return;
  char* mine = arena + shared_bytes + (size_t)c * cta_bytes;
  unsigned gen = 0;
  for (int oi = 0; oi < n; ++oi) {
    const obk::Opt o = opts[oi];
    if (wide_mode(o, split_x) != MODE) continue;  // another instantiation prices it
    int rc = check_option(o, true);
    double ask = dnan(), bid = dnan();
    obk::Stats st;
    st.upts = st.wpts = st.zpts = 0;
    st.zmax_level = 0;
    obk::GroupLay S;
    obk::Lay Lp;
    if (rc == obk::ST_OK && (!obk::carve_group_shared(arena, shared_bytes, o.N, 2 * (o.N + 2), S) ||
                             !obk::carve(mine, cta_bytes, o.N, 16, Lp)))
      rc = obk::ST_CAPACITY;
    if (rc == obk::ST_OK) {
      obk::TcGroup<obk::BlockTeam<kGroupNW>> g(bt, o, Lp, S, G, c);
      obk::TcTrap<obk::BlockTeam<kGroupNW>> tr(bt, o, Lp, S);
      obk::TcSplit<obk::BlockTeam<kGroupNW>> sp(bt, o, Lp, S, G, c);
      rc = g.begin();
      if (rc == obk::ST_OK && !grid_barrier(gs, gen, wait_ns)) rc = ST_TIMEOUT;
      for (int t = o.N; t >= 0 && rc == obk::ST_OK;) {
        // a light level (few points a CTA, small nodes) goes down kTrapD levels in one
        // trapezoid round
        const int B = t + 1;
        const int zb = __ldcg(&S.off[B & 1][2 * (B + 1)]);
        if constexpr (MODE == WIDE_TRAP) {
          if (zb <= kTrapPoints * G && zb <= kTrapColumnPoints * (B + 1)) {
            rc = trap_round(tr, B, G, c, gs, gen, wait_ns, s_cnt, s_cnt2, st, t);
            continue;
          }
        }
        if constexpr (MODE == WIDE_SPLIT) {
          // split the nodes when the largest union of two successors exceeds a share by more
          // than the split's own cost (two more grid barriers and the boundary exchanges)
          if (threadIdx.x == 0) s_max = 0;
          __syncthreads();
          const int* so = S.off[B & 1];
          int m = 0;
          for (int k = threadIdx.x; k < 2 * (B + 1); k += blockDim.x) {
            const int d = __ldcg(&so[k + 1]) - __ldcg(&so[k]);
            m = d > m ? d : m;
          }
          atomicMax(&s_max, m);
          __syncthreads();
          if (split_x < 0.0 || 2LL * s_max * G > 2LL * zb + (long long)kSplitExtraPoints * G) {
            rc = split_level(sp, t, G, c, gs, gen, wait_ns, s_cnt, st);
            --t;
            continue;
          }
        }
        const bool ok = g.compute(t);
        if (threadIdx.x == 0) gs->cnt[t & 1][c] = ok ? g.ztot : -1;
        if (!grid_barrier(gs, gen, wait_ns)) { rc = ST_TIMEOUT; break; }
        int bad = 0;
        for (int k = threadIdx.x; k < G; k += blockDim.x) {
          s_cnt[k] = __ldcg(&gs->cnt[t & 1][k]);
          if (s_cnt[k] < 0) bad = 1;
        }
        if (__syncthreads_or(bad)) { rc = obk::ST_CAPACITY; break; }
        if (!g.publish(t, s_cnt)) { rc = obk::ST_CAPACITY; break; }
        if (!grid_barrier(gs, gen, wait_ns)) { rc = ST_TIMEOUT; break; }
        --t;
      }
      if (rc == obk::ST_OK && c == 0) g.root(ask, bid);
      const obk::Stats gst = g.R.st;
      st.upts += gst.upts;
      st.wpts += gst.wpts;
      st.zpts += gst.zpts;
      if (gst.zmax_level > st.zmax_level) st.zmax_level = gst.zmax_level;
    }
    if (threadIdx.x == 0) {
      if (rc == obk::ST_OK) {
        atomicAdd(&ds->upts, (unsigned long long)st.upts);
        atomicAdd(&ds->wpts, (unsigned long long)st.wpts);
        atomicAdd(&ds->zpts, (unsigned long long)st.zpts);
      }
      if (c == 0) {
        out[2 * oi] = rc ? dnan() : ask;
        out[2 * oi + 1] = rc ? dnan() : bid;
        if (status) status[oi] = rc;
        atomicAdd(&ds->options, 1ULL);
        if (rc == obk::ST_OK) {
          const unsigned long long N = (unsigned long long)o.N;
          atomicAdd(&ds->node_updates, (N + 1) * (N + 2) / 2);
          atomicMax(&ds->max_level, st.zmax_level);
        } else {
          atomicAdd(&ds->failed, 1);
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ CRR on the whole GPU
// Each option in turn on every SM.  The levels advance in tiles of kCrrD levels: CTA c
// takes the tiles of kCrrLen nodes of level T - D from level T's nodes [a, a + kCrrLen + D]
// (its own nodes plus the D-node halo to the right that the recursion reaches), runs the
// D levels in shared memory (the valid region shrinks by one node a level), writes its
// kCrrLen nodes, and all CTAs meet at a grid barrier before the next tile of levels.  The
// exercise table and the leaves are laid out by all CTAs first.
constexpr int kCrrThreads = 256;
constexpr int kCrrD = 64;                       // levels per tile
constexpr int kCrrLen = kCrrThreads - kCrrD;    // nodes a CTA finishes per tile

__global__ void __launch_bounds__(kCrrThreads, 1) k_crr_group(
    const obk::Opt* __restrict__ opts, int n, double* out, int* status, double* buf, size_t buf_doubles,
    GroupState* gs, unsigned long long wait_ns) {
  __shared__ double X[2][kCrrThreads + 1];
  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x;
  unsigned gen = 0;
  for (int oi = 0; oi < n; ++oi) {
    const obk::Opt o = opts[oi];
    int rc = check_option(o, false);
    double res = dnan();
    const int N = o.N;
    if (rc == obk::ST_OK && 4 * (size_t)N + 3 > buf_doubles) rc = obk::ST_CAPACITY;
    const double dt = o.T / N;
    const double u = exp(o.sigma * sqrt(dt));
    const double d = 1.0 / u;
    const double r = exp(o.R * dt);
    if (rc == obk::ST_OK && !(d < r && r < u)) rc = obk::ST_ARBITRAGE;
    if (rc == obk::ST_OK) {
      const double p = (r - d) / (u - d);
      const double pu = p / r, pd = (1.0 - p) / r;
      double* P = buf;  // P[e + N], e = -N..N
      double* Vin = buf + 2 * (size_t)N + 1;
      double* Vout = Vin + N + 1;
      const int stride = G * kCrrThreads;
      for (int e = c * kCrrThreads + tid; e <= 2 * N; e += stride) P[e] = crr_payoff(o, o.S0 * pow(u, (double)(e - N)));
      if (!grid_barrier(gs, gen, wait_ns)) rc = ST_TIMEOUT;
      if (rc == obk::ST_OK) {
        for (int j = c * kCrrThreads + tid; j <= N; j += stride) Vin[j] = P[2 * j];
        if (!grid_barrier(gs, gen, wait_ns)) rc = ST_TIMEOUT;
      }
      int T = N;
      while (rc == obk::ST_OK && T > 0) {
        const int D = T < kCrrD ? T : kCrrD;
        const int Wt = T - D + 1;  // nodes of level T - D
        const int tiles = (Wt + kCrrLen - 1) / kCrrLen;
        for (int tile = c; tile < tiles; tile += G) {
          const int a = tile * kCrrLen;
          for (int k = tid; k <= kCrrThreads; k += kCrrThreads) X[0][k] = (a + k <= T) ? __ldcg(&Vin[a + k]) : 0.0;
          __syncthreads();
          int cur = 0;
          for (int l = 1; l <= D; ++l) {
            const int t = T - l;
            if (tid < kCrrLen + D - l && a + tid <= t)
              X[cur ^ 1][tid] = crr_step(pu, pd, X[cur][tid + 1], X[cur][tid], P[2 * (a + tid) - t + N]);
            __syncthreads();
            cur ^= 1;
          }
          if (tid < kCrrLen && a + tid < Wt) Vout[a + tid] = X[cur][tid];
          __syncthreads();
        }
        if (!grid_barrier(gs, gen, wait_ns)) { rc = ST_TIMEOUT; break; }
        double* tmp = Vin; Vin = Vout; Vout = tmp;
        T -= D;
      }
      if (rc == obk::ST_OK) res = __ldcg(&Vin[0]);
    }
    if (c == 0 && tid == 0) {
      out[oi] = res;
      if (status) status[oi] = rc;
    }
    // every CTA is done with buf before the next option lays out its table
    if (!grid_barrier(gs, gen, wait_ns) && c == 0 && tid == 0 && rc == obk::ST_OK && status) status[oi] = ST_TIMEOUT;
  }
}

cudaError_t crr_group_occupancy(int* per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_crr_group, kCrrThreads, 0);
}

cudaError_t launch_crr_group(int G, cudaStream_t s, const obk::Opt* opts, int n, double* out, int* status,
                             double* buf, size_t buf_doubles, GroupState* gs, unsigned long long wait_ns) {
  void* args[] = {(void*)&opts, (void*)&n, (void*)&out, (void*)&status, (void*)&buf, (void*)&buf_doubles,
                  (void*)&gs, (void*)&wait_ns};
  return cudaLaunchCooperativeKernel((const void*)k_crr_group, dim3(G), dim3(kCrrThreads), args, 0, s);
}

cudaError_t group_occupancy(int* per_sm) {
  int a = 0, b = 0, d = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_tc_group<WIDE_TRAP>, 32 * kGroupNW, 0);
  if (e != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_tc_group<WIDE_SPLIT>, 32 * kGroupNW, 0)) !=
      cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, k_tc_group<WIDE_NODES>, 32 * kGroupNW, 0)) !=
      cudaSuccess)
    return e;
  *per_sm = a < b ? a : b;
  if (d < *per_sm) *per_sm = d;
  return cudaSuccess;
}

cudaError_t launch_group(int G, cudaStream_t s, const obk::Opt* opts, int n, double* out, int* status,
                         char* arena, size_t shared_bytes, size_t cta_bytes, GroupState* gs, DevStats* ds,
                         unsigned long long wait_ns, int skip_cta, double split_x) {
  void* args[] = {(void*)&opts, (void*)&n, (void*)&out, (void*)&status, (void*)&arena,
                  (void*)&shared_bytes, (void*)&cta_bytes, (void*)&gs, (void*)&ds, (void*)&wait_ns,
                  (void*)&skip_cta, (void*)&split_x};
  // one launch per wide_mode; the grid barrier's state starts from zero for each launch
  const void* kern[3] = {(const void*)k_tc_group<WIDE_TRAP>, (const void*)k_tc_group<WIDE_SPLIT>,
                         (const void*)k_tc_group<WIDE_NODES>};
  cudaError_t e = cudaSuccess;
  for (int m = 0; m < 3; ++m) {
    if (m > 0 && (e = cudaMemsetAsync(gs, 0, sizeof(GroupState), s)) != cudaSuccess) return e;
    if ((e = cudaLaunchCooperativeKernel(kern[m], dim3(G), dim3(32 * kGroupNW), args, 0, s)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

}  // namespace obl
