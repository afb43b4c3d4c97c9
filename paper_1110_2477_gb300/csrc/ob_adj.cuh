// ob_adj.cuh -- reverse-mode derivatives of ask and bid with respect to
// (S0, K, sigma, R, T, k): the adjoint of the induction in ob_tc.cuh.
//
// The breakpoint structure is held fixed (the derivative of the piecewise linear
// recursion on the branch the prices take).  Every piece of every node function is a
// line c + s y (in the level's future-value units), and each step of the induction
// takes the pieces of its result from the lines of its inputs or makes them from those
// lines:
//   - pass 1 (w = max of the successors): every piece of w is a piece of one successor;
//   - pass 3 (restriction and exercise): every piece of z is a piece of w, a line of
//     slope -S^a (-S^b) through the point of w where the running minimum of
//     g = w + S^a y (h = w + S^b y) is attained, or a branch of the expense function u.
// So the adjoint carries, per piece, the adjoints of (c, s) -- never of breakpoint
// positions, which move fast where two lines cross at a shallow angle while the
// functions do not.  At a running minimum, on point y* of w between the lines P and Q,
//   g* = (1 - mu) (c_P + (s_P + S) y*) + mu (c_Q + (s_Q + S) y*),  mu = (s_P + S)/(s_P - s_Q),
// is the derivative of the value with the crossing of P and Q moving; at an interior
// minimum mu lies in [0, 1] because the slopes of g on the two sides bracket zero
// (points that coincide with y* to within rounding are resolved by the lines' slopes).
//
// Levels are swept from the root (t = 0) back to the leaves (t = N+1).  The adjoint of
// level t needs a record of the forward level step t: for every point of w its y, slope,
// node and the successor piece it follows, for every point of z the line it follows
// (pass 2 notes where each running minimum is attained).  When the records of all levels
// fit the scratch, the forward pass keeps them (full mode).  Otherwise it keeps the level
// functions at checkpoints every s = ceil(sqrt(N+2)) levels, and each segment between two
// checkpoints is recomputed once with its records before its adjoint levels run.  An
// adjoint level is two scatter loops: the adjoints of z_t's lines go onto w's lines and
// the node constants, then those of w's lines onto level t+1's lines.  Node constants
// (S^a lambda, S^b lambda, xi lambda of every node) are chained to the six parameters in
// closed form.
#pragma once
#include "ob_tc.cuh"

namespace obk {

enum { P_S0 = 0, P_K = 1, P_SIG = 2, P_R = 3, P_T = 4, P_KC = 5, NPAR = 6 };

struct LvRef {
  long long d;  // first double of the level in the store (Y, then F, then S, np each)
  long long o;  // first int of its node offsets
  int np;       // points
};

// Where the record of one level lies in the record store: rd + d (wY, then wS; wtot each)
// and ri + i (wN, wsrc: wtot each; zsrc: ztot; wtail, ztail: 2(t+1) each).
struct LvRec {
  long long d, i;
  int wtot, ztot;
};

struct AdjLay {
  double* sd;       // level store: points
  long long sd_cap;
  int* so;          // level store: node offsets
  long long so_cap;
  LvRef* ref;       // [N+2]
  double *pc[2], *ps[2];  // adjoints of (c, s) of the piece right of each point, two levels [cap]
  double *tc[2], *ts[2];  // ... and of each node's left tail [2(N+2)]
  double *wc, *ws;        // adjoints of the pieces of w right of each point [cap]
  double *wtc, *wts;      // ... and of w's left tails [2(N+1)]
  double *nSa, *nSb, *nXi;  // adjoints of each node's S^a lambda, S^b lambda, xi lambda [2(N+1)]
  int* wsrc;              // pass 1: the successor piece each piece of w follows [cap]
  unsigned* zsrc;         // pass 3: the line each piece of z follows (KW..KU4 codes) [cap]
  int* wtail;             // [2(N+1)] the same for the left tails
  unsigned* ztail;
  int *argA, *argB;       // pass 2: where the running minima of g and h are attained [cap]
  int cap;
  // record store: per level of the segment being swept, what its adjoint needs of the
  // forward level step (y, slope and node of every point of w, and the four codes)
  LvRec* rec;             // [N+2]
  double* rd;             // wY, wS per level
  long long rd_cap;
  int* ri;                // wN, wsrc, zsrc, wtail, ztail per level
  long long ri_cap;
};

// Split an arena between the pricing arrays (cap points each), the adjoint arrays, the
// level store and the record store (full: records of every level, and a level store for
// the leaves and the root only).  Returns false if it does not fit.
OB_HD bool carve_greeks(char* base, size_t bytes, int N, int min_cap, Lay& L, AdjLay& A,
                        bool full = false) {
  const size_t nodes = 2 * ((size_t)N + 2);
  const size_t node_arrays = 4 * al256(sizeof(double) * nodes) + 5 * al256(sizeof(double) * nodes) +
                             2 * al256(sizeof(int) * nodes);
  const size_t nb = node_bytes(N) + 40 * 256 + al256(sizeof(LvRef) * ((size_t)N + 2)) +
                    al256(sizeof(LvRec) * ((size_t)N + 2)) + node_arrays;
  if (bytes < nb) return false;
  const size_t per = ELEM_BYTES + 6 * sizeof(double) + 4 * sizeof(int);
  size_t cap = (size_t)((double)(bytes - nb) * 0.35) / per;
  if (cap > 0x3fffffff) cap = 0x3fffffff;
  if ((long long)cap < (long long)min_cap) return false;
  char* p = carve_cap(base, N, cap, L);
  auto take = [&](size_t sz) { char* r = p; p += al256(sz); return r; };
  A.ref = (LvRef*)take(sizeof(LvRef) * ((size_t)N + 2));
  A.rec = (LvRec*)take(sizeof(LvRec) * ((size_t)N + 2));
  for (int b = 0; b < 2; ++b) {
    A.pc[b] = (double*)take(sizeof(double) * cap);
    A.ps[b] = (double*)take(sizeof(double) * cap);
    A.tc[b] = (double*)take(sizeof(double) * nodes);
    A.ts[b] = (double*)take(sizeof(double) * nodes);
  }
  A.wc = (double*)take(sizeof(double) * cap);
  A.ws = (double*)take(sizeof(double) * cap);
  A.wtc = (double*)take(sizeof(double) * nodes);
  A.wts = (double*)take(sizeof(double) * nodes);
  A.nSa = (double*)take(sizeof(double) * nodes);
  A.nSb = (double*)take(sizeof(double) * nodes);
  A.nXi = (double*)take(sizeof(double) * nodes);
  A.wsrc = (int*)take(sizeof(int) * cap);
  A.zsrc = (unsigned*)take(sizeof(unsigned) * cap);
  A.wtail = (int*)take(sizeof(int) * nodes);
  A.ztail = (unsigned*)take(sizeof(unsigned) * nodes);
  A.argA = (int*)take(sizeof(int) * cap);
  A.argB = (int*)take(sizeof(int) * cap);
  A.cap = (int)cap;
  if ((size_t)(p - base) + 4096 > bytes) return false;
  const size_t rest = bytes - (size_t)(p - base) - 512;
  const int s = (int)ceil(sqrt((double)N + 2.0));
  // offsets: every stored level needs at most 2(N+2)+1 ints; at most 2s+4 levels live
  const size_t so_ints = (size_t)(2 * s + 4) * (2 * ((size_t)N + 2) + 1);
  if (rest < so_ints * sizeof(int) + 4096) return false;
  A.so = (int*)take(sizeof(int) * so_ints);
  A.so_cap = (long long)so_ints;
  // the rest: 45 % level store (checkpoints and the segment's levels, 24 bytes a point),
  // 55 % record store (the segment's records, 16 + 12 bytes a point of w, 4 of z); in full
  // mode 10 % and 90 %
  const size_t left = bytes - (size_t)(p - base) - 1024;
  const size_t lv = (size_t)((double)left * (full ? 0.10 : 0.45)) & ~(size_t)255;
  A.sd = (double*)take(lv);
  A.sd_cap = (long long)(lv / sizeof(double));
  const size_t rdb = ((left - lv) * 4 / 7) & ~(size_t)255;  // doubles: 16 of every 28 bytes
  A.rd = (double*)take(rdb);
  A.rd_cap = (long long)(rdb / sizeof(double));
  A.ri = (int*)p;
  A.ri_cap = (long long)((bytes - (size_t)(p - base)) / sizeof(int)) - 64;
  return A.sd_cap > 0 && A.ri_cap > 0;
}

OB_HD void atomic_add(double* a, double v) {
#if defined(__CUDA_ARCH__)
  if (v != 0.0) atomicAdd(a, v);
#else
  if (v != 0.0) {  // host builds of this header: compare-and-swap loop
    long long expect = __atomic_load_n((long long*)a, __ATOMIC_RELAXED);
    for (;;) {
      const long long want = dbits(bitsd(expect) + v);
      if (__atomic_compare_exchange_n((long long*)a, &expect, want, false, __ATOMIC_RELAXED,
                                      __ATOMIC_RELAXED))
        break;
    }
  }
#endif
}

template <class Team>
struct TcAdj {
  TcRun<Team>& R;
  const Team& tm;
  const Opt& o;
  const Lay& L;
  const AdjLay& A;
  int N;
  double g[2][NPAR];     // this lane's share of d ask / d theta (g[0]) and d bid / d theta (g[1])
  long long sd_top, so_top;
  long long rd_top = 0, ri_top = 0;

  // the record of one level (see LvRec)
  struct RecView {
    const double *wY, *wS;
    const int *wN, *wsrc;
    const unsigned* zsrc;
    const int* wtail;
    const unsigned* ztail;
    int wtot, ztot;
  };
  OB_HD RecView view(int t) const {
    const LvRec r = A.rec[t];
    const int nodes = 2 * (t + 1);
    RecView v;
    v.wY = A.rd + r.d;
    v.wS = v.wY + r.wtot;
    v.wN = A.ri + r.i;
    v.wsrc = v.wN + r.wtot;
    v.zsrc = (const unsigned*)(v.wsrc + r.wtot);
    v.wtail = (const int*)(v.zsrc + r.ztot);
    v.ztail = (const unsigned*)(v.wtail + nodes);
    v.wtot = r.wtot;
    v.ztot = r.ztot;
    return v;
  }
  // keep what the adjoint of level t needs from the level step just run
  OB_HD bool rec_store(int t, int wtot, int ztot) {
    const int nodes = 2 * (t + 1);
    const long long nd = 2LL * wtot, ni = 2LL * wtot + ztot + 2LL * nodes;
    if (rd_top + nd > A.rd_cap || ri_top + ni > A.ri_cap) return false;
    A.rec[t] = LvRec{rd_top, ri_top, wtot, ztot};
    rd_top += nd;
    ri_top += ni;
    double* wY = A.rd + A.rec[t].d;
    double* wS = wY + wtot;
    int* wN = A.ri + A.rec[t].i;
    int* wsrc = wN + wtot;
    unsigned* zsrc = (unsigned*)(wsrc + wtot);
    int* wtail = (int*)(zsrc + ztot);
    unsigned* ztail = (unsigned*)(wtail + nodes);
    for (int i = tm.lane(); i < wtot; i += Team::W) {
      wY[i] = L.wY[i];
      wS[i] = L.wS[i];
      wN[i] = L.wN[i];
      wsrc[i] = A.wsrc[i];
    }
    for (int i = tm.lane(); i < ztot; i += Team::W) zsrc[i] = A.zsrc[i];
    for (int n = tm.lane(); n < nodes; n += Team::W) {
      wtail[n] = A.wtail[n];
      ztail[n] = A.ztail[n];
    }
    tm.sync();
    return true;
  }
  // level t from level t+1 (the in-views) into its bank, recording for its adjoint
  OB_HD bool level_recorded(int t) {
    const int bt = t & 1;
    R.outY = L.zY[bt]; R.outF = L.zF[bt]; R.outS = L.zS[bt]; R.outOff = L.off[bt];
    R.outCap = L.capZ;
    R.node_table(t + 1);
    R.node_table(t);
    tm.sync();
    int wtot, utot, ztot;
    if (!R.template pass1<true>(t, wtot, utot, 0, -1, A.wsrc, A.wtail)) return false;
    if (wtot > A.cap) return false;
    R.template pass2<true>(t, wtot, A.argA, A.argB);
    if (!R.template pass3<true>(t, wtot, ztot, 0, A.zsrc, A.ztail, A.argA, A.argB)) return false;
    tm.sync();
    return rec_store(t, wtot, ztot);
  }

  OB_HD TcAdj(TcRun<Team>& R_, const AdjLay& A_)
      : R(R_), tm(R_.tm), o(R_.o), L(R_.L), A(A_), N(R_.N) {
    for (int p = 0; p < 2; ++p)
      for (int k = 0; k < NPAR; ++k) g[p][k] = 0.0;
    sd_top = so_top = 0;
  }

  // ---------------------------------------------------------------- node constants
  // Adds dSa * d(S^a lambda)/d theta + dSb * d(S^b lambda)/d theta + dxi * d(xi lambda)/d theta
  // of node (t, j) to party p's gradient.
  OB_HD void acc_node(int t, int j, int p, double dSa, double dSb, double dxi) {
    if (dSa == 0.0 && dSb == 0.0 && dxi == 0.0) return;
    const int e = 2 * j - t;
    const double S = L.Stab[e + N + 1];
    const double lam = L.lam[t];
    const double kt = (t == 0) ? 0.0 : o.k;
    const double rootTN = sqrt(o.T / N);
    double dlnS[NPAR] = {1.0 / o.S0, 0.0, e * rootTN, 0.0, e * o.sigma / (2.0 * sqrt(o.T * N)), 0.0};
    double dlnL[NPAR] = {0.0, 0.0, 0.0, (double)(N + 1 - t) * o.T / N, (double)(N + 1 - t) * o.R / N, 0.0};
    const double Sl = S * lam;
    const double Sa = Sl * (1.0 + kt), Sb = Sl * (1.0 - kt);
    double xi_raw, dxi_dS = 0.0, dxi_dK = 0.0;
    if (o.payoff == PAY_PUT) { xi_raw = o.K; dxi_dK = 1.0; }
    else if (o.payoff == PAY_CALL) { xi_raw = -o.K; dxi_dK = -1.0; }
    else {
      const bool aK = S > o.K, aK2 = S > o.K2;
      xi_raw = (aK ? S - o.K : 0.0) - (aK2 ? S - o.K2 : 0.0);
      dxi_dS = (aK ? 1.0 : 0.0) - (aK2 ? 1.0 : 0.0);
      dxi_dK = (aK ? -1.0 : 0.0) + (aK2 ? 1.0 : 0.0);
    }
    const double xi = xi_raw * lam;
    for (int k = 0; k < NPAR; ++k) {
      const double dl = dlnS[k] + dlnL[k];
      double dSa_k = Sa * dl, dSb_k = Sb * dl;
      if (k == P_KC && t > 0) { dSa_k += Sl; dSb_k -= Sl; }
      double dxi_k = lam * dxi_dS * S * dlnS[k] + xi * dlnL[k];
      if (k == P_K) dxi_k += lam * dxi_dK;
      g[p][k] += dSa * dSa_k + dSb * dSb_k + dxi * dxi_k;
    }
  }

  // ---------------------------------------------------------------- level store
  OB_HD bool store_alloc(int t, int np) {
    const long long need_d = 3LL * np, need_o = 2LL * (t + 1) + 1;
    if (sd_top + need_d > A.sd_cap || so_top + need_o > A.so_cap) return false;
    A.ref[t] = LvRef{sd_top, so_top, np};
    sd_top += need_d;
    so_top += need_o;
    return true;
  }
  OB_HD void in_from_store(int t) {
    const LvRef r = A.ref[t];
    R.inY = A.sd + r.d;
    R.inF = R.inY + r.np;
    R.inS = R.inF + r.np;
    R.inOff = A.so + r.o;
  }
  // copy level t from its bank into the store
  OB_HD bool store_from_bank(int t) {
    const int b = t & 1;
    const int np = L.off[b][2 * (t + 1)];
    if (!store_alloc(t, np)) return false;
    const LvRef r = A.ref[t];
    for (int i = tm.lane(); i < np; i += Team::W) {
      A.sd[r.d + i] = L.zY[b][i];
      A.sd[r.d + np + i] = L.zF[b][i];
      A.sd[r.d + 2 * np + i] = L.zS[b][i];
    }
    for (int n = tm.lane(); n <= 2 * (t + 1); n += Team::W) A.so[r.o + n] = L.off[b][n];
    tm.sync();
    return true;
  }
  // compute level t into its bank from the level t+1 the in-views point at
  OB_HD bool level_to_bank(int t) {
    const int bt = t & 1;
    R.outY = L.zY[bt]; R.outF = L.zF[bt]; R.outS = L.zS[bt]; R.outOff = L.off[bt];
    R.outCap = L.capZ;
    R.node_table(t + 1);  // the successors' tails (its bank may hold another level by now)
    R.node_table(t);
    tm.sync();
    int wtot, utot, ztot;
    if (!R.pass1(t, wtot, utot)) return false;
    R.pass2(t, wtot);
    if (!R.pass3(t, wtot, ztot)) return false;
    return true;
  }

  // ---------------------------------------------------------------- adjoint of pass 3
  // The lines of w around point a (a point where a running minimum is attained): the
  // piece left of it (the piece right of a - 1, or w's left tail if a starts its node)
  // and the piece right of it.  Slopes: wS, or the tail's -S^a of the level-(t+1) node
  // it comes from.
  OB_HD double left_slope(int t, const RecView& V, int a, int node, bool first) const {
    if (!first) return V.wS[a - 1];
    const int code = V.wtail[node];  // -1 - (level-(t+1) node)
    const int n1 = -1 - code, W1 = t + 2;
    const int j1 = n1 >= W1 ? n1 - W1 : n1;
    return -L.nt[(t + 1) & 1][4 * j1];
  }

  // Line adjoint (cb, sb) of a piece of z at level t, following the line of `code`.
  OB_HD void pull_z(int t, const RecView& V, unsigned code, double cb, double sb) {
    if (cb == 0.0 && sb == 0.0) return;
    const int kind = (int)(code >> KSHIFT);
    int a = (int)(code & KMASK);
    const int W0 = t + 1;
    const int node = V.wN[a];
    const int p = node >= W0 ? 1 : 0;
    const int j = node - p * W0;
    const double* nt = L.nt[t & 1];
    if (kind == KW) {
      atomic_add(&A.wc[a], cb);
      atomic_add(&A.ws[a], sb);
      return;
    }
    if (kind == KA || kind == KB) {
      const double S = nt[4 * j + (kind == KA ? 0 : 1)];
      // resolve points that coincide with y_a to within rounding by the lines' slopes
      const double tol = 1e-12 * fmax(1.0, fabs(V.wY[a]));
      for (int it = 0; it < 64; ++it) {
        const bool last = (a + 1 >= V.wtot) || V.wN[a + 1] != node;
        if (last || !(V.wS[a + 1] + S < 0.0) || V.wY[a + 1] - V.wY[a] > tol) break;
        ++a;
      }
      for (int it = 0; it < 64; ++it) {
        const bool first = (a == 0) || V.wN[a - 1] != node;
        if (first || !(V.wS[a - 1] + S > 0.0) || V.wY[a] - V.wY[a - 1] > tol) break;
        --a;
      }
      const bool first = (a == 0) || V.wN[a - 1] != node;
      const double sP = left_slope(t, V, a, node, first), sQ = V.wS[a];
      const double mu = (sP == sQ) ? 0.0 : (sP + S) / (sP - sQ);
      const double ys = V.wY[a];
      if (first) {
        atomic_add(&A.wtc[node], (1.0 - mu) * cb);
        atomic_add(&A.wts[node], (1.0 - mu) * ys * cb);
      } else {
        atomic_add(&A.wc[a - 1], (1.0 - mu) * cb);
        atomic_add(&A.ws[a - 1], (1.0 - mu) * ys * cb);
      }
      atomic_add(&A.wc[a], mu * cb);
      atomic_add(&A.ws[a], mu * ys * cb);
      // the S y* term of the minimum and the line's slope -S
      atomic_add(kind == KA ? &A.nSa[node] : &A.nSb[node], ys * cb - sb);
      return;
    }
    // a branch of u: c = vu + S yu, s = -S, vu = xi (seller) or -xi (buyer), yu = kink of u
    const bool seller = (p == 0);
    const double yu = seller ? (double)R.zeta : -(double)R.zeta;
    atomic_add(&A.nXi[node], seller ? cb : -cb);
    atomic_add(kind == KU3 ? &A.nSa[node] : &A.nSb[node], yu * cb - sb);
  }

  // z_t's line adjoints (pc, ps per point; tc, ts per node) onto w's lines and the node
  // constants of level t
  OB_HD void scatter_z(int t, const RecView& V, const double* pc, const double* ps, const double* tc,
                       const double* ts) {
    const int nNodes = 2 * (t + 1);
    for (int i = tm.lane(); i < V.ztot; i += Team::W) pull_z(t, V, V.zsrc[i], pc[i], ps[i]);
    for (int n = tm.lane(); n < nNodes; n += Team::W) pull_z(t, V, V.ztail[n], tc[n], ts[n]);
    tm.sync();
    const int W0 = t + 1;
    for (int n = tm.lane(); n < nNodes; n += Team::W) {
      const int p = n >= W0 ? 1 : 0;
      acc_node(t, n - p * W0, p, A.nSa[n], A.nSb[n], A.nXi[n]);
    }
  }

  // w's line adjoints onto the lines of level t+1 (pc1, ps1 per point; tc1, ts1 per node)
  OB_HD void scatter_w(int t, const RecView& V, double* pc1, double* ps1, double* tc1, double* ts1) {
    for (int i = tm.lane(); i < V.wtot; i += Team::W) {
      const double cb = A.wc[i], sb = A.ws[i];
      if (cb == 0.0 && sb == 0.0) continue;
      const int code = V.wsrc[i];
      if (code >= 0) {
        atomic_add(&pc1[code], cb);
        atomic_add(&ps1[code], sb);
      } else {
        atomic_add(&tc1[-1 - code], cb);
        atomic_add(&ts1[-1 - code], sb);
      }
    }
    for (int n = tm.lane(); n < 2 * (t + 1); n += Team::W) {
      const double cb = A.wtc[n], sb = A.wts[n];
      if (cb == 0.0 && sb == 0.0) continue;
      const int code = V.wtail[n];
      atomic_add(&tc1[-1 - code], cb);
      atomic_add(&ts1[-1 - code], sb);
    }
    tm.sync();
  }

  OB_HD void zero(double* a, int n) {
    for (int i = tm.lane(); i < n; i += Team::W) a[i] = 0.0;
  }

  // ---------------------------------------------------------------- driver
  // Returns a status; on success lane 0's gA / gB hold d ask / d theta and d bid / d theta.
  OB_HD int run(double& ask, double& bid, double* gA, double* gB, bool full = false) {
    const int lane = tm.lane();
    ask = bid = 0.0;
    const double dt = o.T / N;
    const double u = exp(o.sigma * sqrt(dt));
    const double r = exp(o.R * dt);
    const double d = 1.0 / u;
    if (!(d < r && r < u)) return ST_ARBITRAGE;
    for (int e = lane; e < 2 * N + 3; e += Team::W) L.Stab[e] = o.S0 * pow(u, (double)(e - (N + 1)));
    for (int t = lane; t <= N + 1; t += Team::W) L.lam[t] = pow(r, (double)(N + 1 - t));
    tm.sync();
    const int s = (int)ceil(sqrt((double)N + 2.0));
    auto is_ckpt = [&](int t) { return ((N + 1 - t) % s) == 0; };
    // leaves, stored as the first checkpoint
    {
      const int b = (N + 1) & 1, W = N + 2;
      R.node_table(N + 1);
      tm.sync();
      for (int n = lane; n < 2 * W; n += Team::W) {
        const int j = n >= W ? n - W : n;
        L.off[b][n] = n;
        L.zY[b][n] = 0.0;
        L.zF[b][n] = 0.0;
        L.zS[b][n] = -L.nt[b][4 * j + 1];
      }
      if (lane == 0) L.off[b][2 * W] = 2 * W;
      tm.sync();
      if (!store_from_bank(N + 1)) return ST_CAPACITY;
    }
    // forward, keeping checkpoints (full mode: none; its one segment below is the forward)
    for (int t = N; !full && t >= 0; --t) {
      const int b1 = (t + 1) & 1;
      R.inY = L.zY[b1]; R.inF = L.zF[b1]; R.inS = L.zS[b1]; R.inOff = L.off[b1];
      if (!level_to_bank(t)) return ST_CAPACITY;
      if (is_ckpt(t) && !store_from_bank(t)) return ST_CAPACITY;
    }
    const long long ckpt_sd = sd_top, ckpt_so = so_top;
    // reverse sweep, one segment per checkpoint, from the root upward (full mode: one
    // segment from the leaves, whose levels are not stored, only counted, but the root)
    int cur = 0;  // adjoint bank of the current level
    int lo = 0;   // lowest level whose functions the next segment must provide
    bool seeded = false;
    for (int c = 0; c <= N + 1; ++c) {
      if (full ? c != N + 1 : !is_ckpt(c)) continue;
      if (c < lo) continue;
      // recompute levels c-1 .. lo from the checkpoint c (kept in the store after the checkpoints)
      sd_top = ckpt_sd;
      so_top = ckpt_so;
      rd_top = ri_top = 0;
      for (int t = c - 1; t >= lo; --t) {
        if (full) {
          const int b1 = (t + 1) & 1;
          R.inY = L.zY[b1]; R.inF = L.zF[b1]; R.inS = L.zS[b1]; R.inOff = L.off[b1];
        } else {
          in_from_store(t + 1);
        }
        if (!level_recorded(t)) return ST_CAPACITY;
        if (full && t > 0) {
          if (lane == 0) A.ref[t] = LvRef{0, 0, L.off[t & 1][2 * (t + 1)]};  // its point count only
        } else if (!store_from_bank(t)) {
          return ST_CAPACITY;
        }
      }
      if (!seeded && c > 0) {  // root: the value at y = 0 of the piece right of every point <= 0
        seeded = true;
        const LvRef r0 = A.ref[0];
        const double* Y0 = A.sd + r0.d;
        const double* F0 = Y0 + r0.np;
        const double* S0v = F0 + r0.np;
        const int* off0 = A.so + r0.o;
        zero(A.pc[cur], r0.np); zero(A.ps[cur], r0.np);
        zero(A.tc[cur], 2); zero(A.ts[cur], 2);
        tm.sync();
        const double lam0 = L.lam[0];
        double vals[2];
        for (int p = 0; p < 2; ++p) {
          const int b = off0[p], e = off0[p + 1];
          const double sc = (p == 0 ? 1.0 : -1.0) / lam0;
          const double tailL = -L.nt[0][0];
          double v;
          if (e <= b) { vals[p] = 0.0; continue; }
          int k = b;  // first point right of 0
          while (k < e && kle(Y0[k], 0.0)) ++k;
          if (k == b) {
            v = F0[b] + tailL * (0.0 - Y0[b]);
            if (lane == 0) A.tc[cur][p] += sc;
          } else {
            v = F0[k - 1] + S0v[k - 1] * (0.0 - Y0[k - 1]);
            if (lane == 0) A.pc[cur][k - 1] += sc;
          }
          vals[p] = (p == 0) ? v / lam0 : -v / lam0;  // ask, then bid (as the pricing path)
        }
        ask = vals[0];
        bid = vals[1];
        tm.sync();
        if (lane == 0) {  // the division by lambda_0 = r^(N+1)
          const double dl_R = (double)(N + 1) * o.T / N, dl_T = (double)(N + 1) * o.R / N;
          g[0][P_R] -= ask * dl_R; g[0][P_T] -= ask * dl_T;
          g[1][P_R] -= bid * dl_R; g[1][P_T] -= bid * dl_T;
        }
      }
      // adjoint levels lo .. c-1 (each needs level t+1 <= c), from the records
      for (int t = lo; t <= c - 1; ++t) {
        R.node_table(t + 1);
        R.node_table(t);
        tm.sync();
        const RecView V = view(t);
        const int nNodes = 2 * (t + 1), nNodes1 = 2 * (t + 2);
        const int nxt = cur ^ 1;
        const int np1 = A.ref[t + 1].np;
        if (np1 > A.cap || V.wtot > A.cap) return ST_CAPACITY;
        zero(A.wc, V.wtot); zero(A.ws, V.wtot);
        zero(A.wtc, nNodes); zero(A.wts, nNodes);
        zero(A.nSa, nNodes); zero(A.nSb, nNodes); zero(A.nXi, nNodes);
        zero(A.pc[nxt], np1); zero(A.ps[nxt], np1);
        zero(A.tc[nxt], nNodes1); zero(A.ts[nxt], nNodes1);
        tm.sync();
        scatter_z(t, V, A.pc[cur], A.ps[cur], A.tc[cur], A.ts[cur]);
        tm.sync();
        scatter_w(t, V, A.pc[nxt], A.ps[nxt], A.tc[nxt], A.ts[nxt]);
        cur = nxt;
      }
      lo = c;
    }
    // leaves: their lines are c = 0 with slopes -S^a (tail) and -S^b (the point's piece)
    {
      const int W = N + 2;
      for (int n = lane; n < 2 * W; n += Team::W) {
        const int p = n >= W ? 1 : 0;
        const int j = n - p * W;
        acc_node(N + 1, j, p, -A.ts[cur][n], -A.ps[cur][n], 0.0);
      }
    }
    for (int p = 0; p < 2; ++p)
      for (int k = 0; k < NPAR; ++k) {
        const double v = tm.sum(g[p][k]);
        if (lane == 0) (p == 0 ? gA : gB)[k] = v;
      }
    return ST_OK;
  }
};

}  // namespace obk
