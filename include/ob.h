/* ob.h -- C ABI of the GB300 ask/bid pricer for American options under
 * proportional transaction costs.
 *
 * What is computed (Zhang, Roux & Zastawniak, "Parallel Binomial American
 * Option Pricing with (and without) Transaction Costs", 2011):
 *   - Section 4.1: a recombining binomial tree with N steps,
 *     u = exp(sigma*sqrt(T/N)), d = 1/u, r = exp(R*T/N), plus an extra time
 *     instant N+1 whose N+2 nodes carry the payoff (0,0); no transaction costs
 *     at t = 0.
 *   - Section 3: stock bought at S^a = (1+k)S and sold at S^b = (1-k)S; the
 *     seller's expense function (Eq. 1) and the buyer's (Eq. 6); the backward
 *     induction w_t = max of the successors' functions, discount by r,
 *     restriction of the slopes to [-S^a_t, -S^b_t], then z_t = max(u_t, v_t)
 *     (seller, Roux & Zastawniak Algorithm 3.1) or z_t = min(u_t, v_t) (buyer,
 *     Algorithm 3.5).  ask = z_0(0), bid = -z'_0(0).
 *   - Section 3 (first paragraph) and the Appendix: without costs the same
 *     numbers equal the plain CRR American price, computed by the scalar
 *     recursion pi_t = max(P_t, (p pi^u + (1-p) pi^d)/r) over N levels.
 * All arithmetic is IEEE binary64.
 *
 * Threading and ordering: calls may come from any host thread and on any
 * stream.  A call that uses the library's scratch pool on a device enqueues
 * under that device's mutex and orders its device work behind the previous
 * pooled call's (it waits on an event the previous call recorded, then
 * records its own), so calls on different streams never overlap in the pool.
 * While the caller's stream is being captured into a CUDA graph this ordering
 * is skipped (an event recorded outside a capture cannot be waited on inside
 * it); such callers order their calls themselves.  Kernels run
 * asynchronously on the given stream.  Growing the pool synchronises the
 * device.  ob_price_ask_bid_noalloc uses a fixed array of its own instead of
 * the pool: overlapping calls of it race.
 */
#ifndef OB_H_
#define OB_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One option, 64 bytes, host byte order, tightly packed.  Field meaning:
 *   S0     stock price at t = 0 (> 0)
 *   K      strike (>= 0); for the bull spread the long call's strike
 *   K2     bull spread only: the short call's strike (>= K); ignored otherwise
 *   sigma  volatility (> 0), R continuously compounded annual rate (finite),
 *   T      expiry in years (> 0), k cost rate, 0 <= k < 1
 *   N      time steps (>= 1)
 *   payoff OB_PUT: payoff process (K, -1), physical delivery (Section 3);
 *          OB_CALL: (-K, +1), physical delivery;
 *          OB_SPREAD: cash-settled bull spread, xi = (S-K)^+ - (S-K2)^+,
 *          zeta = 0 (Section 5). */
typedef struct {
  double S0, K, K2, sigma, R, T, k;
  int32_t N, payoff;
} ob_option_t;

enum { OB_PUT = 0, OB_CALL = 1, OB_SPREAD = 2 };

/* Status / return codes. */
enum {
  OB_OK = 0,
  OB_ERR_ARG = -1,       /* a parameter outside the ranges above, or bad pointers/sizes */
  OB_ERR_ARBITRAGE = -2, /* d < r < u fails, so the tree model admits arbitrage */
  OB_ERR_CAPACITY = -3,  /* the option's piecewise-linear functions outgrew the scratch pool */
  OB_ERR_TIMEOUT = -4,   /* a bounded device wait expired */
  OB_ERR_CUDA = -5,      /* a CUDA runtime call failed (see ob_last_cuda_error) */
  OB_ERR_NOMEM = -6      /* the scratch pool could not be allocated */
};

/* Ask and bid of n_options options (Section 3, Algorithms 3.1 / 3.5).
 *   params  DEVICE pointer, n_options records, read only.
 *   out     DEVICE pointer, 2*n_options doubles: out[2i] = ask, out[2i+1] = bid.
 *   status  DEVICE pointer to n_options int32 (may be NULL): OB_OK or the
 *           option's error code; an option that fails leaves NaN in out and
 *           does not stop the others.
 *   stream  cudaStream_t (NULL = legacy default stream).
 * Batched form: one persistent launch whose CTAs take options from a device
 * queue, costliest first (work stealing), each option on a whole-CTA team (one
 * 512-thread CTA per SM by default, see ob_configure); once the options left
 * are predicted to cost less than 4 % of the mean work per SM
 * (OB_SPLIT_FACTOR), each 16-warp CTA splits into two 8-warp teams that take
 * options independently (two options per SM); options whose functions
 * outgrow a CTA's scratch are retried by follow-up launches with larger
 * scratch, on the same stream, without returning to the host.  The launch
 * sequence is captured in a CUDA graph per (params, n_options, out, status)
 * and replayed when the same buffers come back (it reads their current
 * contents).  Asynchronous: returns OB_OK once the work is enqueued, or an
 * error code (nothing enqueued) for bad arguments, allocation failure or a
 * launch error.  The library's scratch pool is allocated on the first call on
 * a device (cudaMalloc, so make that call before any stream capture) and kept
 * until ob_release(). */
int ob_price_ask_bid(const ob_option_t* params, int64_t n_options, double* out, int32_t* status,
                     void* stream);

/* ob_price_ask_bid plus the hedge at the root of each option (Section 3: the
 * rebalancing at t = 0, where there are no costs).  A portfolio covers the
 * seller from t = 1 on iff, after moving its stock holding to y', its cash
 * lies above w_0/r at y'; v_0(0) = min over y' of w_0(y')/r + S0 y'.
 *   hedge   DEVICE pointer, 4*n_options doubles:
 *           hedge[4i]   the seller's stock holding y* after rebalancing at t = 0
 *                       from no stock (the y' attaining v_0(0); the rightmost
 *                       among equal minima),
 *           hedge[4i+1] the buyer's (the same for the buyer's functions),
 *           hedge[4i+2] 1 when immediate exercise sets the ask (u_0(0) > v_0(0)),
 *                       else 0,
 *           hedge[4i+3] 1 when the buyer does better exercising at once
 *                       (u_0(0) < v_0(0)), else 0;
 *           NaN for an option whose status is not OB_OK.
 * Without costs (k = 0) y* is the CRR delta at t = 0 for the seller and its
 * negative for the buyer.  Same launch sequence, graph caching and ordering as
 * ob_price_ask_bid (hedge joins the graph key); the fused on-chip level step is
 * not used by this call.  Returns OB_ERR_ARG when hedge is NULL. */
int ob_price_ask_bid_hedge(const ob_option_t* params, int64_t n_options, double* out, int32_t* status,
                           double* hedge, void* stream);

/* The hedge along one path of the tree per option (Section 3, the rebalancing of
 * ob_price_ask_bid_hedge made at every node the path visits): at level t the
 * hedger moves its stock holding from the one it arrived with (no stock before
 * t = 0) to the y' attaining v_t(y) = min over y' of w_t(y')/r + theta_t(y' - y),
 * theta_t buying at S^a = (1+k) S and selling at S^b = (1-k) S (k = 0 at t = 0);
 * the rightmost y' among equal minima.  The buyer stops at the first level
 * where exercising with the holding it arrived with costs less than keeping
 * the hedge, u_t(y) < v_t(y) (Eq. 6's expense for the buyer).
 *   params  DEVICE pointer, n_options options (as for ob_price_ask_bid).
 *   moves   DEVICE pointer, n_options * stride int8: moves[i*stride + t] for
 *           t < N_i is the move from level t to t+1 (non-zero up, 0 down);
 *           the path's node at level t is the number of up moves before t.
 *   stride  row length of moves, 1 <= stride; every N_i <= stride (an option
 *           with N_i > stride gets OB_ERR_ARG in status).
 *   out     DEVICE pointer, 2*n_options doubles: ask and bid, equal bit for bit
 *           to ob_price_ask_bid's.
 *   hold    DEVICE pointer, n_options * (stride+1) * 2 doubles:
 *           hold[(i*(stride+1) + t)*2]     the seller's holding after
 *                                          rebalancing at level t (t <= N_i),
 *           hold[(i*(stride+1) + t)*2 + 1] the buyer's, NaN from its stopping
 *                                          level on;
 *           NaN for t > N_i and for an option whose status is not OB_OK.
 *   cash    DEVICE pointer or NULL, same layout as hold: each party's cash after
 *           rebalancing at level t, in time-t money, of the self-financing
 *           portfolio that starts at t = 0 with no stock and the ask (seller)
 *           or minus the bid (buyer, who borrows it to buy the option):
 *           x_t = r x_{t-1} - theta_t(y_t - y_{t-1}).  Along any path the
 *           seller's portfolio can settle an exercise at every level and its
 *           stock at N+1, and the buyer's can settle the buyer's exercise at
 *           its stopping level (or its stock at N+1); NaN where hold is.
 *   stop    DEVICE pointer, n_options int32: the buyer's stopping level, -1 if
 *           it never stops (or the status is not OB_OK).
 *   status  DEVICE pointer or NULL, n_options int32 (as for ob_price_ask_bid).
 * One 16-warp CTA team per option, up to one per SM, taking the options from a
 * device queue (the costliest first for batches up to 8192 options, in index
 * order above), with 128 MiB of scratch each (OB_PATH_MB): three quarters for
 * the level arrays, one quarter for w_t of the path's nodes.  An option that
 * outgrows either part is retried by a second launch of one CTA team with the
 * whole pool, on the same stream; one that outgrows that too gets
 * OB_ERR_CAPACITY and NaN.  Same pool, serialisation and call ordering as
 * ob_price_ask_bid.  Returns OB_ERR_ARG on a NULL pointer (status may be NULL)
 * or stride outside [1, 2^26]. */
int ob_hedge_path(const ob_option_t* params, int64_t n_options, const int8_t* moves, int64_t stride,
                  double* out, double* hold, double* cash, int32_t* stop, int32_t* status, void* stream);

/* The plain form of the same computation: one warp per option, options taken
 * in index order with a static assignment, no queue and no retry (an option
 * that outgrows its warp's scratch gets OB_ERR_CAPACITY).  Arguments and
 * results as for ob_price_ask_bid.  This is the single-option kernel the
 * batched form is compared against. */
int ob_price_ask_bid_plain(const ob_option_t* params, int64_t n_options, double* out,
                           int32_t* status, void* stream);

/* Fixed-scratch form of ob_price_ask_bid, for callers that cannot allocate
 * device memory at call time: code running inside a memory budget that is
 * already fully handed out, callers that must not touch the allocator while
 * other work is in flight, or hosts whose process-wide allocation policy
 * forbids cudaMalloc after start-up.  (The paper has no counterpart; this is an
 * interface convenience.)
 *
 * It prices with the same kernels as ob_price_ask_bid, but all of its scratch
 * lives in one file-scope device array of OB_NOALLOC_SCRATCH_BYTES that every
 * device holds from the moment the library is loaded until the process exits;
 * the call itself allocates and frees nothing.  The caller passes params, out
 * and status (device pointers, as for ob_price_ask_bid).
 *   - n_options must not exceed OB_NOALLOC_MAX_OPTIONS; larger batches are
 *     rejected with OB_ERR_ARG and nothing is enqueued.
 *   - An option whose functions outgrow the fixed scratch gets
 *     OB_ERR_CAPACITY in status (NaN in out); the others complete.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress), so make that first call before any stream
 *     capture.
 *   - Every call on a device shares the array and resets its counters on the
 *     given stream; calls whose work overlaps on the GPU (different streams,
 *     or different host threads without ordering) race on it and must be
 *     serialised by the caller. */
#define OB_NOALLOC_SCRATCH_BYTES (64u << 20)
#define OB_NOALLOC_MAX_OPTIONS 4096
int ob_price_ask_bid_noalloc(const ob_option_t* params, int64_t n_options, double* out,
                             int32_t* status, void* stream);

/* Derivatives of ask and bid (the adjoint of the induction), with the prices.
 *   params  DEVICE pointer, n_options records.
 *   out     DEVICE pointer, 2*n_options doubles (ask, bid), as ob_price_ask_bid.
 *   grad    DEVICE pointer, 12*n_options doubles: grad[12i + 0..5] = d ask / d(S0, K,
 *           sigma, R, T, k), grad[12i + 6..11] = d bid / d(the same).
 *   status  DEVICE pointer to n_options int32, or NULL.
 * Meaning: the derivative of the piecewise-linear recursion along the branch the
 * prices take (breakpoint structure held fixed); at a kink of the price in a
 * parameter (an exercise boundary, a breakpoint appearing) it is one of the
 * one-sided derivatives.  d/dK of the bull spread moves both strikes (fixed
 * width); d/dT changes the step T/N with N fixed; at k = 0, d/dk is the
 * right-hand derivative.  Method: reverse mode over the levels, root to leaves.
 * The forward pass keeps a record of every level step (which line each piece
 * follows) when the option's predicted records fit its scratch; otherwise it
 * keeps the level functions at checkpoints every ceil(sqrt(N+2)) levels and
 * recomputes each segment once, with its records.  One 16-warp CTA team per
 * option (OB_GREEKS_WARPS=8 for 8-warp teams), one CTA per SM, options taken
 * from a device queue; follow-up launches with larger scratch (and checkpoints)
 * for options that outgrow a CTA's share of the pool.  Asynchronous on stream. */
int ob_greeks(const ob_option_t* params, int64_t n_options, double* out, double* grad,
              int32_t* status, void* stream);

/* Whole-GPU form, for large single options (N in the thousands): the options are
 * priced one after another, each on every SM at once.  One CTA per SM; at each
 * level the CTAs split the nodes by their merged successor breakpoints (whole
 * nodes, G equal shares), run the same element-wise passes as ob_price_ask_bid
 * into private scratch, then place their breakpoints in the shared level; two
 * grid barriers per level.  Puts, and calls with k <= sigma sqrt(T/N), take their
 * light levels (at most 128 points per CTA) eight at a time: each CTA works on a
 * window of columns with a halo of its neighbour's (Section 4.2's blocks of
 * levels), two barriers per round.  Calls and spreads with k > 6 sigma sqrt(T/N)
 * split their largest nodes over the CTAs on the levels where a node outgrows a
 * share (four barriers per level).  Three cooperative launches per call, one per
 * kind of option.  Results are bitwise equal to ob_price_ask_bid.  Arguments,
 * ownership and statuses as ob_price_ask_bid; a barrier wait longer than 10 s
 * gives OB_ERR_TIMEOUT for the option in progress and every later option of its
 * launch; a level that outgrows the shared scratch (1/8 of the pool) gives
 * OB_ERR_CAPACITY. */
int ob_price_ask_bid_wide(const ob_option_t* params, int64_t n_options, double* out,
                          int32_t* status, void* stream);

/* Plain CRR American price without transaction costs (the Appendix): the
 * scalar recursion over N levels, no extra level; k is ignored.
 *   out  DEVICE pointer, n_options doubles.  Other arguments as above. */
int ob_crr_american(const ob_option_t* params, int64_t n_options, double* out, int32_t* status,
                    void* stream);

/* Whole-GPU form of ob_crr_american, for large single options (N in the
 * thousands and up): the options are priced one after another, each on every SM
 * at once.  One cooperative launch of a CTA per SM; the levels advance in tiles
 * of 64 levels: each CTA takes 192 nodes of the tile's last level together with
 * the 64-node halo the recursion reaches from them, runs the 64 levels in shared
 * memory, writes its nodes back, and all CTAs meet at a grid barrier.  The same
 * node update as ob_crr_american, so the results agree bit for bit.  Arguments
 * and statuses as ob_crr_american; a barrier wait longer than 10 s gives
 * OB_ERR_TIMEOUT for the option in progress and the later ones; an option needs
 * 4N+3 doubles of the scratch pool (OB_ERR_CAPACITY beyond). */
int ob_crr_american_wide(const ob_option_t* params, int64_t n_options, double* out, int32_t* status,
                         void* stream);

/* Host-buffer convenience form of ob_price_ask_bid: params, out (2*n) and
 * status (n, may be NULL) are HOST pointers; the call copies the inputs to
 * the device, runs the batched form on an internal stream, copies the results
 * back and returns after they have arrived.  Pinned host memory makes the
 * copies faster but is not required. */
int ob_price_ask_bid_host(const ob_option_t* params, int64_t n_options, double* out,
                          int32_t* status);

/* Counters of the most recent ob_price_ask_bid / _plain call on the current
 * device.  Call after that work has completed (synchronise its stream). */
typedef struct {
  int64_t options;        /* options processed (any status) */
  int64_t node_updates;   /* (N+1)(N+2)/2 summed over successfully priced options */
  int64_t u_points;       /* successor breakpoints merged into the maxima w, both parties */
  int64_t w_points;       /* breakpoints of all successor maxima w, both parties */
  int64_t z_points;       /* breakpoints of all node functions z, both parties */
  int32_t max_level_points; /* largest number of breakpoints held by one tree level */
  int32_t retried;        /* options that needed a follow-up launch with larger scratch */
  int32_t failed;         /* options with a nonzero status */
  int32_t tiers;          /* launches enqueued by the call */
  int32_t graph;          /* batched form: 0 direct launches, 1 captured into a new CUDA
                             graph and launched, 2 replay of a cached graph */
  int32_t team_warps;     /* warps per CTA team of the batched form */
  int32_t chip_points;    /* batched form: points of w each CTA team keeps in shared memory
                             (the fused level step; 0: w in the global scratch) */
  int32_t half_teams;     /* batched form: 1 when 16-warp CTAs split into two 8-warp teams for
                             the light options (OB_SPLIT_FACTOR > 0 and no fused step), else 0 */
} ob_stats_t;
int ob_get_stats(ob_stats_t* host_out);

/* Configuration of the batched form on the current device.
 *   team_warps  warps per CTA team (4, 8, 12 or 16; the grid is 16 / team_warps CTAs
 *               per SM (one for 12), each with 1 / (CTAs) of the scratch pool as its
 *               breakpoint capacity); 0 keeps the current value (default 16).
 *   use_graphs  1: ob_price_ask_bid captures its launch sequence (queue reset, cost
 *               order, persistent kernel, two follow-up tiers) into a CUDA graph per
 *               (params, n, out, status) key, keeps the last 4, and replays a graph
 *               when the key repeats; 0: plain launches; -1 keeps (default 1).
 *   chip_points the fused level step of 16- and 8-warp teams: passes 1-3 run per chunk
 *               of whole nodes with w, the keys of g and h and their running minima in
 *               shared memory (a chunk holds up to this many points of w, 60 bytes each;
 *               nodes beyond it run on the global scratch); -1 as many as the CTA's
 *               shared memory holds, 0 off (default; measured slower on the 4096-option
 *               batch, since the shared memory is taken from the L1 cache), -2 keeps.
 *               Results do not depend on it (bitwise).
 * Drops the cached graphs.  Returns OB_ERR_ARG for another team width. */
int ob_configure(int32_t team_warps, int32_t use_graphs, int32_t chip_points);

/* Autotuner of the batched form: times seven configurations -- 16-warp teams that split
 * into two 8-warp teams for the light options, 16-warp teams throughout, team widths 12,
 * 8, 4 warps (hence the CTA size, the registers per thread and the per-CTA breakpoint
 * capacity) with w in the global scratch, then the fused level step with w on chip (all
 * the shared memory a CTA can take) for 16 and 8 warps -- on a sample of the given
 * options (every (n_options / sample)-th option; sample <= 0 or >= n_options: all of
 * them), one warm-up run and one timed run each, with CUDA events on stream, and keeps
 * the fastest for later calls (a candidate replaces an earlier one only when it is more
 * than 1 % faster).  Synchronous.  params is a DEVICE pointer as in
 * ob_price_ask_bid.  team_warps_out and chip_out (HOST, may be NULL) receive the
 * choice (chip_out: on-chip points per CTA, 0 for none; ob_stats_t.half_teams tells the
 * first two apart); ms_out (HOST, 7 floats, may be NULL) the timed milliseconds in the
 * order above. */
int ob_autotune(const ob_option_t* params, int64_t n_options, int64_t sample, void* stream,
                int32_t* team_warps_out, int32_t* chip_out, float* ms_out);

/* Release the current device's scratch pool (synchronises the device). */
int ob_release(void);

/* Human-readable text of a status code; never NULL. */
const char* ob_strerror(int code);

/* The CUDA error string of the last OB_ERR_CUDA returned on this thread. */
const char* ob_last_cuda_error(void);

/* Measurement helper (the paper has no counterpart): the device's FP64 fused
 * multiply-add throughput, the denominator of the FP64 rooflines the benchmark
 * reports.  One launch of 8 CTAs of 256 threads per SM, each thread running 8
 * independent chains of `iters` DFMAs (2 flops each), timed with CUDA events on
 * stream; three runs, the fastest of the last two is kept.  Synchronous.
 *   tflops_out  HOST pointer: measured TFLOP/s.
 *   ms_out      HOST pointer (may be NULL): the kept run's milliseconds.
 * Returns OB_ERR_ARG for iters <= 0 or a NULL tflops_out. */
int ob_fp64_peak(int64_t iters, void* stream, double* tflops_out, double* ms_out);

#ifdef __cplusplus
}
#endif

#endif /* OB_H_ */
