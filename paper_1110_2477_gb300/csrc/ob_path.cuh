// ob_path.cuh -- the hedge along a path of the tree (Section 3): the level passes of
// ob_tc.cuh for one option on a team, keeping w_t of the nodes a given path visits, then the
// rebalancing at every node of the path.  A portfolio covers the seller from t+1 on iff,
// after moving its stock holding from y to y', its cash lies above w_t/r at y'; the cheapest
// such move attains v_t(y) = inf over y' of w_t(y')/r + theta_t(y' - y).  Host and device
// code (the host build runs it with a one-lane team in the CPU tests).
#pragma once
#include "ob_tc.cuh"

namespace obk {

// w_t of one path node, kept during the induction: points [off, off + m) of the store (y,
// value, right slope; future-value units of level t, i.e. w_t/r scaled by lambda_t) and the
// slope of its left tail.
struct PathLv {
  long long off;
  int m;
  double sL;
};

// The holding y' that attains min over y' of F(y') + (y' >= y0 ? sa : sb)(y' - y0) for the
// piecewise-linear F of m points (Y, V, right slopes S; left tail slope sL): the minimum lies
// at a breakpoint of F or at y0.  Candidates in increasing order; among equal values the
// rightmost.  Writes the minimum to vmin.
OB_HD double rebalance_to(const double* Y, const double* V, const double* S, int m, double sL, double sa,
                          double sb, double y0, double& vmin) {
  double best_y = 0.0, best_v = 0.0;
  bool have = false;
  bool y0_done = false;
  auto consider = [&](double c, double fc) {
    const double v = fc + (c >= y0 ? sa : sb) * (c - y0);
    if (!have || v <= best_v) {
      best_v = v;
      best_y = c;
      have = true;
    }
  };
  for (int k = 0; k < m; ++k) {
    if (!y0_done && y0 < Y[k]) {  // y0 before breakpoint k: on the piece left of it
      const double f0 = (k == 0) ? V[0] + sL * (y0 - Y[0]) : V[k - 1] + S[k - 1] * (y0 - Y[k - 1]);
      consider(y0, f0);
      y0_done = true;
    }
    consider(Y[k], V[k]);
  }
  if (!y0_done) consider(y0, V[m - 1] + S[m - 1] * (y0 - Y[m - 1]));
  vmin = best_v;
  return best_y;
}

// One option (already checked: N >= 1, parameters in range): the induction of TcRun::run with
// the path's w_t kept, then the rebalancing along the path by lane 0.  moves[t] (t < N):
// non-zero up, 0 down.  hold and cash (may be null): 2 (N+1) doubles.  The cash of a self-financing portfolio is carried in future-value
// units, where it changes only by the cost of each rebalancing: X_t = X_{t-1} - theta_t
// lambda_t (y_t - y_{t-1}), X_{-1} = ask lambda_0 (seller) or -bid lambda_0 (buyer); the
// cash in time-t money is X_t / lambda_t.
template <class Team>
OB_HD int path_one(const Team& tm, const Opt& o, const int8_t* moves, char* slice, size_t bytes, double& ask,
                   double& bid, double* hold, double* cash, int& stop) {
  const double qnan = bitsd(0x7ff8000000000000LL);
  ask = bid = qnan;
  stop = -1;
  const int N = o.N, lane = tm.lane();
  // the level arrays in the first three quarters, the path store in the rest
  const size_t lay_bytes = (bytes / 4 * 3) & ~(size_t)255;
  Lay L;
  if (!carve(slice, lay_bytes, N, 2 * (N + 2), L)) return ST_CAPACITY;
  const size_t lv_bytes = al256(sizeof(PathLv) * 2 * ((size_t)N + 1));
  if (bytes < lay_bytes + lv_bytes + 256) return ST_CAPACITY;
  PathLv* lv = (PathLv*)(slice + lay_bytes);  // [2 (N+1)]: level t, party p at 2t + p
  double* store = (double*)(slice + lay_bytes + lv_bytes);
  const long long store_cap = (long long)((bytes - lay_bytes - lv_bytes) / sizeof(double)) - 8;
  TcRun<Team> R(tm, o, L);
  const double dt = o.T / N;
  const double u = exp(o.sigma * sqrt(dt));
  const double r = exp(o.R * dt);
  const double d = 1.0 / u;
  if (!(d < r && r < u)) return ST_ARBITRAGE;
  for (int e = lane; e < 2 * N + 3; e += Team::W) L.Stab[e] = o.S0 * pow(u, (double)(e - (N + 1)));
  for (int t = lane; t <= N + 1; t += Team::W) L.lam[t] = pow(r, (double)(N + 1 - t));
  int ups = 0;  // j_N: the up moves of the whole path
  for (int b = 0; b < N; b += Team::W) ups += tm.count(b + lane < N && moves[b + lane] != 0);
  tm.sync();
  {  // level N+1: payoff (0,0) for both parties
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
  }
  if (2 * (N + 2) > L.capZ) return ST_CAPACITY;
  long long used = 0;
  int j = ups;  // the path's node at the current level
  for (int t = N; t >= 0; --t) {
    if (t < N) j -= moves[t] != 0 ? 1 : 0;
    R.use_banks(t);
    R.node_table(t);
    tm.sync();
    int wtot = 0, ztot = 0, utot = 0;
    if (!R.pass1(t, wtot, utot)) return ST_CAPACITY;
    R.pass2(t, wtot);
    if (!R.pass3(t, wtot, ztot)) return ST_CAPACITY;
    // keep w of the path's seller node j and buyer node t + 1 + j (w is ordered by node):
    // the first point of each node and of the next one, four binary searches on the points'
    // node index, one per lane, into the four slots past the store
    const double* nt1 = L.nt[(t + 1) & 1];
    long long* bound = (long long*)(store + store_cap);
    for (int k = lane; k < 4; k += Team::W) {
      const int node = (k >> 1) * (t + 1) + j + (k & 1);
      int a = 0, b = wtot;
      while (a < b) {
        const int mid = (a + b) >> 1;
        if (L.wN[mid] < node) a = mid + 1;
        else b = mid;
      }
      bound[k] = a;
    }
    tm.sync();
    for (int p = 0; p < 2; ++p) {
      const int lo = (int)bound[2 * p], hi = (int)bound[2 * p + 1];
      const int m = hi - lo;
      if (m < 1 || used + 3LL * m > store_cap) return ST_CAPACITY;
      for (int i = lane; i < m; i += Team::W) {
        store[used + i] = L.wY[lo + i];
        store[used + m + i] = L.wF[lo + i];
        store[used + 2 * m + i] = L.wS[lo + i];
      }
      if (lane == 0) lv[2 * t + p] = PathLv{used, m, -nt1[4 * (j + 1)]};  // the up successor's -S^a
      used += 3LL * m;
    }
    tm.sync();
  }
  const double lam0 = L.lam[0];
  const double z0s = R.root_value(0), z0b = R.root_value(1);
  ask = z0s / lam0;
  bid = -z0b / lam0;
  if (lane == 0) {  // the rebalancing along the path
    double ys = 0.0, yb = 0.0, Xs = z0s, Xb = z0b;
    int jj = 0;
    for (int t = 0; t <= N; ++t) {
      if (t > 0) jj += moves[t - 1] != 0 ? 1 : 0;
      const double S = L.Stab[2 * jj - t + N + 1];
      const double Sl = S * L.lam[t];
      const double kt = (t == 0) ? 0.0 : o.k;
      const double sa = Sl * (1.0 + kt), sb = Sl * (1.0 - kt);
      const PathLv a = lv[2 * t], b = lv[2 * t + 1];
      double v;
      const double y1 =
          rebalance_to(store + a.off, store + a.off + a.m, store + a.off + 2 * a.m, a.m, a.sL, sa, sb, ys, v);
      Xs -= (y1 >= ys ? sa : sb) * (y1 - ys);
      ys = y1;
      hold[2 * t] = ys;
      if (cash) cash[2 * t] = Xs / L.lam[t];
      if (stop >= 0) {
        hold[2 * t + 1] = qnan;
        if (cash) cash[2 * t + 1] = qnan;
        continue;
      }
      const double y = rebalance_to(store + b.off, store + b.off + b.m, store + b.off + 2 * b.m, b.m, b.sL, sa,
                                    sb, yb, v);
      // the buyer's expense of exercising now with holding yb (Eq. 6), future-value units
      double xi;
      if (o.payoff == PAY_PUT) xi = o.K;
      else if (o.payoff == PAY_CALL) xi = -o.K;
      else xi = fmax(S - o.K, 0.0) - fmax(S - o.K2, 0.0);
      const double zeta = (o.payoff == PAY_PUT) ? -1.0 : (o.payoff == PAY_CALL ? 1.0 : 0.0);
      const double q = yb + zeta;
      const double ue = -xi * L.lam[t] + (q < 0.0 ? -q * sa : -q * sb);
      if (ue < v) {
        stop = t;
        hold[2 * t + 1] = qnan;
        if (cash) cash[2 * t + 1] = qnan;
      } else {
        Xb -= (y >= yb ? sa : sb) * (y - yb);
        hold[2 * t + 1] = yb = y;
        if (cash) cash[2 * t + 1] = Xb / L.lam[t];
      }
    }
  }
  tm.sync();
  return ST_OK;
}

}  // namespace obk
