// ob_oracle.cpp -- TEST INFRASTRUCTURE, not part of the product path.
//
// A plain, slow, obviously-correct CPU implementation of what the GPU library
// computes, written from the paper (N. Zhang, A. Roux, T. Zastawniak,
// "Parallel Binomial American Option Pricing with (and without) Transaction
// Costs", 2011).  Only the tests, the package smoke check and the benchmark's
// CPU-baseline leg may load it.  It shares no code, header or table with the
// CUDA library.
//
// What it computes
//  * Section 4.1: the binomial model u = exp(sigma*sqrt(T/N)), d = 1/u,
//    r = exp(R*T/N), an extra time instant N+1 whose N+2 nodes carry the
//    payoff (0,0), and no transaction costs at t = 0.
//  * Section 3: bid/ask stock prices S^a = (1+k)S, S^b = (1-k)S; the seller's
//    expense function u_t (Eq. 1) and the buyer's (Eq. 6); and the backward
//    induction that builds, at every node, w_t = max of the two successor z's,
//    the discounted w_t/r, its slope restriction v_t to [-S^a_t, -S^b_t], and
//    z_t = max(u_t, v_t) for the seller (ask = z_0(0)) or z_t = min(u_t, v_t)
//    for the buyer (bid = -z'_0(0)).  These are Roux & Zastawniak's
//    Algorithms 3.1 and 3.5 as the paper sketches them.
//  * Section 3 (first paragraph) and the Appendix: the plain CRR recursion
//    pi_t = max(P_t, (p pi^u + (1-p) pi^d)/r) without costs, with no extra
//    level, and its European counterpart (no early exercise).
//  * Forward-mode dual numbers through the same induction give the
//    derivatives of ask and bid with respect to (S0, K, sigma, R, T, k).
//  * Section 4.2, Algorithm 1: the paper's own parallel scheme (blocks of
//    levels, regions A and B, signals between neighbouring threads, a barrier
//    per round) driving the same node steps on host threads, as a CPU
//    comparator; its results are bitwise the serial ones.
//
// Readings of the paper taken here:
//  * "restricting the slopes" of w_t/r to [-S^a_t, -S^b_t] is the
//    inf-convolution v(y) = inf_{y'} [ w(y')/r + theta(y'-y) ], with
//    theta(x) = S^a x for x >= 0 and S^b x for x < 0: the cheapest way to
//    rebalance from stock holding y to y' and then hold a covering position.
//    It is the largest function below w/r whose slopes lie in the window; for
//    the convex seller functions it is a clip of the slopes, for the
//    (non-convex) buyer functions it is computed by two monotone sweeps.
//  * node (t, j) has stock price S_{t,j} = S0 u^(2j-t); its successors are
//    (t+1, j+1) (up) and (t+1, j) (down).
//  * payoffs (xi, zeta): put (K, -1) and call (-K, +1), both physically
//    settled; bull spread cash-settled, xi = (S-K)^+ - (S-K2)^+, zeta = 0.
//
// Representation: a piecewise-linear (PL) function is a strictly increasing
// list of breakpoints y_i with values f_i, plus the slopes of the two tails.
// Every breakpoint kept is a genuine kink: results are simplified
// structurally (a point is dropped when the same input piece continues
// through it), never by a floating-point collinearity test.
//
// Build: g++ -O2 -ffp-contract=off -std=c++17 -shared -fPIC -pthread

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

extern "C" {
// 64-byte option record (same layout as the workload tables).
typedef struct {
  double S0, K, K2, sigma, R, T, k;
  int32_t N, payoff;
} or_option_t;
}

namespace {

enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_ARBITRAGE = -2, OR_ERR_UNBOUNDED = -3,
       OR_ERR_CAPACITY = -4 };
enum { PAY_PUT = 0, PAY_CALL = 1, PAY_SPREAD = 2 };

// ---------------------------------------------------------------- dual numbers
// Value plus its gradient with respect to (S0, K, sigma, R, T, k).
constexpr int NG = 6;
struct Dual {
  double v;
  double g[NG];
  Dual() : v(0) { for (int i = 0; i < NG; ++i) g[i] = 0; }
  Dual(double x) : v(x) { for (int i = 0; i < NG; ++i) g[i] = 0; }
};
inline Dual operator+(const Dual& a, const Dual& b) {
  Dual c; c.v = a.v + b.v; for (int i = 0; i < NG; ++i) c.g[i] = a.g[i] + b.g[i]; return c;
}
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual c; c.v = a.v - b.v; for (int i = 0; i < NG; ++i) c.g[i] = a.g[i] - b.g[i]; return c;
}
inline Dual operator-(const Dual& a) {
  Dual c; c.v = -a.v; for (int i = 0; i < NG; ++i) c.g[i] = -a.g[i]; return c;
}
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual c; c.v = a.v * b.v;
  for (int i = 0; i < NG; ++i) c.g[i] = a.g[i] * b.v + a.v * b.g[i];
  return c;
}
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual c; c.v = a.v / b.v;
  for (int i = 0; i < NG; ++i) c.g[i] = (a.g[i] - c.v * b.g[i]) / b.v;
  return c;
}
inline Dual dexp(const Dual& a) {
  Dual c; c.v = std::exp(a.v); for (int i = 0; i < NG; ++i) c.g[i] = c.v * a.g[i]; return c;
}
inline Dual dsqrt(const Dual& a) {
  Dual c; c.v = std::sqrt(a.v);
  for (int i = 0; i < NG; ++i) c.g[i] = a.g[i] / (2.0 * c.v);
  return c;
}
inline Dual dpowi(const Dual& a, int e) {
  Dual c; c.v = std::pow(a.v, e);
  double dv = (e == 0) ? 0.0 : e * std::pow(a.v, e - 1);
  for (int i = 0; i < NG; ++i) c.g[i] = dv * a.g[i];
  return c;
}
inline double dexp(double a) { return std::exp(a); }
inline double dsqrt(double a) { return std::sqrt(a); }
inline double dpowi(double a, int e) { return std::pow(a, e); }

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }

// ---------------------------------------------------------------- PL functions
template <class T>
struct PL {
  std::vector<T> y, f;  // strictly increasing breakpoints and values
  T sL, sR;             // slopes for y < y.front() and y > y.back()
};

template <class T>
T pl_eval(const PL<T>& F, const T& x) {
  const size_t m = F.y.size();
  const double xv = val(x);
  if (xv <= val(F.y[0])) return F.f[0] + F.sL * (x - F.y[0]);
  if (xv >= val(F.y[m - 1])) return F.f[m - 1] + F.sR * (x - F.y[m - 1]);
  size_t lo = 0, hi = m - 1;  // y[lo] <= x < y[hi]
  while (hi - lo > 1) {
    size_t mid = (lo + hi) / 2;
    if (val(F.y[mid]) <= xv) lo = mid; else hi = mid;
  }
  if (xv == val(F.y[lo])) return F.f[lo];
  T t = (x - F.y[lo]) / (F.y[hi] - F.y[lo]);
  return F.f[lo] + (F.f[hi] - F.f[lo]) * t;
}

// Pointwise max (take_max) or min of F and G.  The union of both breakpoint
// sets is evaluated on both functions; wherever F - G changes sign strictly
// between neighbouring union points (or in a tail) the crossing is inserted.
// owners (optional): for each piece of the result (the left tail, the piece right of each
// breakpoint), 1 if it is a piece of F, 2 if of G.
template <class T>
PL<T> pl_envelope(const PL<T>& F, const PL<T>& G, bool take_max, std::vector<int>* owners = nullptr) {
  enum { OF = 1, OG = 2 };
  struct UP { T y; int iF, iG; };
  std::vector<UP> U;
  size_t i = 0, j = 0;
  const size_t mF = F.y.size(), mG = G.y.size();
  while (i < mF || j < mG) {
    if (j == mG || (i < mF && val(F.y[i]) < val(G.y[j]))) { U.push_back({F.y[i], (int)i, -1}); ++i; }
    else if (i == mF || val(G.y[j]) < val(F.y[i])) { U.push_back({G.y[j], -1, (int)j}); ++j; }
    else { U.push_back({F.y[i], (int)i, (int)j}); ++i; ++j; }
  }
  const size_t n = U.size();
  std::vector<T> a(n), b(n);
  std::vector<int> s(n);  // +1: F wins strictly, -1: G wins strictly, 0: tie
  for (size_t q = 0; q < n; ++q) {
    a[q] = U[q].iF >= 0 ? F.f[U[q].iF] : pl_eval(F, U[q].y);
    b[q] = U[q].iG >= 0 ? G.f[U[q].iG] : pl_eval(G, U[q].y);
    const double av = val(a[q]), bv = val(b[q]);
    s[q] = (av == bv) ? 0 : (((av > bv) == take_max) ? 1 : -1);
  }
  auto owner = [](int sg) { return sg > 0 ? OF : OG; };

  struct OP { T y, f; int iF, iG; };
  std::vector<OP> P;      // candidate output points, in order
  std::vector<int> own;   // own[q]: owner of the segment left of P[q]; own.back(): right tail

  // Left tail: the function with the smaller slope is larger far to the left.
  int farL;
  {
    const double dl = val(F.sL) - val(G.sL);
    if (dl != 0) farL = ((dl < 0) == take_max) ? OF : OG;
    else farL = (s[0] >= 0) ? OF : OG;
  }
  own.push_back(farL);
  if (s[0] != 0 && owner(s[0]) != farL) {
    T h0 = a[0] - b[0];
    T dL = F.sL - G.sL;
    T ys = U[0].y - h0 / dL;
    if (val(ys) < val(U[0].y)) {
      T fs = a[0] + F.sL * (ys - U[0].y);
      P.push_back({ys, fs, -1, -1});
      own.push_back(owner(s[0]));
    }
  }
  for (size_t q = 0; q < n; ++q) {
    P.push_back({U[q].y, (s[q] >= 0 ? a[q] : b[q]), U[q].iF, U[q].iG});
    if (q + 1 == n) break;
    const int sl = s[q], sr = s[q + 1];
    if (sl * sr < 0) {
      T h0 = a[q] - b[q], h1 = a[q + 1] - b[q + 1];
      T t = h0 / (h0 - h1);
      T ys = U[q].y + (U[q + 1].y - U[q].y) * t;
      if (val(ys) > val(U[q].y) && val(ys) < val(U[q + 1].y)) {
        T fs = a[q] + (a[q + 1] - a[q]) * t;
        own.push_back(owner(sl));
        P.push_back({ys, fs, -1, -1});
        own.push_back(owner(sr));
      } else if (val(ys) <= val(U[q].y)) {
        own.push_back(owner(sr));
      } else {
        own.push_back(owner(sl));
      }
    } else {
      const int ss = sl + sr;
      own.push_back(ss > 0 ? OF : (ss < 0 ? OG : OF));
    }
  }
  // Right tail: the function with the larger slope is larger far to the right.
  int farR;
  {
    const double dr = val(F.sR) - val(G.sR);
    if (dr != 0) farR = ((dr > 0) == take_max) ? OF : OG;
    else farR = (s[n - 1] >= 0) ? OF : OG;
  }
  if (s[n - 1] != 0 && owner(s[n - 1]) != farR) {
    T h0 = a[n - 1] - b[n - 1];
    T dR = F.sR - G.sR;
    T ys = U[n - 1].y - h0 / dR;
    if (val(ys) > val(U[n - 1].y)) {
      T fs = a[n - 1] + F.sR * (ys - U[n - 1].y);
      own.push_back(owner(s[n - 1]));
      P.push_back({ys, fs, -1, -1});
    }
  }
  own.push_back(farR);

  PL<T> out;
  out.sL = own.front() == OF ? F.sL : G.sL;
  out.sR = own.back() == OF ? F.sR : G.sR;
  if (owners) owners->assign(1, own.front());
  for (size_t q = 0; q < P.size(); ++q) {
    const int ol = own[q], orr = own[q + 1];
    const bool kink = (ol != orr) || (ol == OF ? P[q].iF >= 0 : P[q].iG >= 0);
    if (kink) {
      out.y.push_back(P[q].y);
      out.f.push_back(P[q].f);
      if (owners) owners->push_back(orr);
    }
  }
  if (out.y.empty()) {
    out.y.push_back(P[0].y);
    out.f.push_back(P[0].f);
    if (owners) owners->push_back(own.back());
  }
  return out;
}

template <class T>
PL<T> pl_div(const PL<T>& F, const T& r) {
  PL<T> out = F;
  for (auto& v : out.f) v = v / r;
  out.sL = F.sL / r;
  out.sR = F.sR / r;
  return out;
}

// Slope restriction v(y) = inf_{y'} [ F(y') + theta(y' - y) ] = min(A(y), B(y)),
//   A(y) = min_{y' >= y} [F(y') + Sa y'] - Sa y   (buy stock, swept from the right)
//   B(y) = min_{y' <= y} [F(y') + Sb y'] - Sb y   (sell stock, swept from the left)
// Each of A, B follows F ("active") or a line of slope -Sa / -Sb ("flat").
// The pieces of a restriction, for the derivatives: for each piece of A and of B (left
// tail first) whether it follows F (ACT) or is a flat line, and for a flat line the
// breakpoint of F where the running minimum it carries is attained; for each piece of V
// whether it is a piece of A (1) or of B (2).
struct RestrictPieces {
  std::vector<int> a_own, a_arg, b_own, b_arg, v_own;
  std::vector<double> a_y, b_y;  // breakpoints of A and B
};

template <class T>
int pl_restrict(const PL<T>& F, const T& Sa, const T& Sb, PL<T>& V, RestrictPieces* rp = nullptr) {
  enum { ACT = 1, FLAT = 2 };
  const size_t m = F.y.size();
  if (val(F.sR) + val(Sa) < 0 || val(F.sL) + val(Sb) > 0) return OR_ERR_UNBOUNDED;
  struct SP { T y, f; int iF; };

  // ---- A: sweep from the right over g = F + Sa*y.
  PL<T> A;
  {
    std::vector<SP> P;     // right-to-left
    std::vector<int> own;  // own[q]: owner of the segment right of P[q] (own[0] = right tail)
    std::vector<int> arg;  // arg[q]: for a flat segment, the breakpoint where its minimum is attained
    own.push_back(ACT);
    arg.push_back(-1);
    T cur = F.f[m - 1] + Sa * F.y[m - 1];
    int cur_i = (int)(m - 1);
    bool act_right = true;  // is M equal to g at the current right end point?
    P.push_back({F.y[m - 1], F.f[m - 1], (int)(m - 1)});
    for (size_t ii = m - 1; ii-- > 0;) {
      T gi = F.f[ii] + Sa * F.y[ii];
      T gr = F.f[ii + 1] + Sa * F.y[ii + 1];
      if (val(gi) >= val(cur)) {
        own.push_back(FLAT); arg.push_back(cur_i);
        P.push_back({F.y[ii], cur - Sa * F.y[ii], (int)ii});
        act_right = false;
      } else if (act_right) {
        own.push_back(ACT); arg.push_back(-1);
        P.push_back({F.y[ii], F.f[ii], (int)ii});
        cur = gi;
        cur_i = (int)ii;
      } else {
        T t = (cur - gi) / (gr - gi);  // g(y*) = cur, measured from y_i
        T ys = F.y[ii] + (F.y[ii + 1] - F.y[ii]) * t;
        if (val(ys) > val(F.y[ii]) && val(ys) < val(F.y[ii + 1])) {
          own.push_back(FLAT); arg.push_back(cur_i);
          P.push_back({ys, cur - Sa * ys, -1});
          own.push_back(ACT); arg.push_back(-1);
        } else if (val(ys) >= val(F.y[ii + 1])) {
          own.push_back(ACT); arg.push_back(-1);
        } else {
          own.push_back(FLAT); arg.push_back(cur_i);
        }
        P.push_back({F.y[ii], F.f[ii], (int)ii});
        cur = gi;
        cur_i = (int)ii;
        act_right = true;
      }
    }
    // left tail: g(y) = g_0 + (sL + Sa)(y - y_0)
    const double slg = val(F.sL) + val(Sa);
    T tailslope;
    if (slg <= 0) {
      own.push_back(FLAT); arg.push_back(cur_i);
      tailslope = -Sa;
    } else if (act_right) {
      own.push_back(ACT); arg.push_back(-1);
      tailslope = F.sL;
    } else {
      T g0 = F.f[0] + Sa * F.y[0];
      T ys = F.y[0] - (g0 - cur) / (F.sL + Sa);
      if (val(ys) < val(F.y[0])) {
        own.push_back(FLAT); arg.push_back(cur_i);
        P.push_back({ys, cur - Sa * ys, -1});
      }
      own.push_back(ACT); arg.push_back(-1);
      tailslope = F.sL;
    }
    // P is right-to-left; own[q] is right of P[q], own[q+1] is left of P[q].
    A.sR = F.sR;  // own[0] == ACT
    A.sL = tailslope;
    std::vector<T> yy, ff;
    std::vector<int> lo, la;  // owner and argument of the piece left of each kept point
    for (size_t q = 0; q < P.size(); ++q) {
      const int orr = own[q], ol = own[q + 1];
      const bool kink = (ol != orr) || (ol == ACT && P[q].iF >= 0);
      if (kink) { yy.push_back(P[q].y); ff.push_back(P[q].f); lo.push_back(ol); la.push_back(arg[q + 1]); }
    }
    if (yy.empty()) {
      yy.push_back(P[0].y); ff.push_back(P[0].f);
      lo.push_back(own.back()); la.push_back(arg.back());
    }
    A.y.assign(yy.rbegin(), yy.rend());
    A.f.assign(ff.rbegin(), ff.rend());
    if (rp) {  // pieces of A from the left: left of each kept point (leftmost first), the right tail
      rp->a_own.assign(lo.rbegin(), lo.rend());
      rp->a_arg.assign(la.rbegin(), la.rend());
      rp->a_own.push_back(own[0]);
      rp->a_arg.push_back(arg[0]);
    }
  }

  // ---- B: sweep from the left over h = F + Sb*y.
  PL<T> B;
  {
    std::vector<SP> P;     // left-to-right
    std::vector<int> own;  // own[q]: owner of the segment left of P[q] (own[0] = left tail)
    std::vector<int> arg;  // arg[q]: for a flat segment, the breakpoint where its minimum is attained
    own.push_back(ACT);
    arg.push_back(-1);
    T cur = F.f[0] + Sb * F.y[0];
    int cur_i = 0;
    bool act_left = true;
    P.push_back({F.y[0], F.f[0], 0});
    for (size_t ii = 1; ii < m; ++ii) {
      T hi = F.f[ii] + Sb * F.y[ii];
      T hl = F.f[ii - 1] + Sb * F.y[ii - 1];
      if (val(hi) >= val(cur)) {
        own.push_back(FLAT); arg.push_back(cur_i);
        P.push_back({F.y[ii], cur - Sb * F.y[ii], (int)ii});
        act_left = false;
      } else if (act_left) {
        own.push_back(ACT); arg.push_back(-1);
        P.push_back({F.y[ii], F.f[ii], (int)ii});
        cur = hi;
        cur_i = (int)ii;
      } else {
        T t = (hl - cur) / (hl - hi);  // h(y*) = cur, measured from y_{i-1}
        T ys = F.y[ii - 1] + (F.y[ii] - F.y[ii - 1]) * t;
        if (val(ys) > val(F.y[ii - 1]) && val(ys) < val(F.y[ii])) {
          own.push_back(FLAT); arg.push_back(cur_i);
          P.push_back({ys, cur - Sb * ys, -1});
          own.push_back(ACT); arg.push_back(-1);
        } else if (val(ys) <= val(F.y[ii - 1])) {
          own.push_back(ACT); arg.push_back(-1);
        } else {
          own.push_back(FLAT); arg.push_back(cur_i);
        }
        P.push_back({F.y[ii], F.f[ii], (int)ii});
        cur = hi;
        cur_i = (int)ii;
        act_left = true;
      }
    }
    const double srh = val(F.sR) + val(Sb);
    T tailslope;
    if (srh >= 0) {
      own.push_back(FLAT); arg.push_back(cur_i);
      tailslope = -Sb;
    } else if (act_left) {
      own.push_back(ACT); arg.push_back(-1);
      tailslope = F.sR;
    } else {
      T hm = F.f[m - 1] + Sb * F.y[m - 1];
      T ys = F.y[m - 1] + (cur - hm) / (F.sR + Sb);
      if (val(ys) > val(F.y[m - 1])) {
        own.push_back(FLAT); arg.push_back(cur_i);
        P.push_back({ys, cur - Sb * ys, -1});
      }
      own.push_back(ACT); arg.push_back(-1);
      tailslope = F.sR;
    }
    B.sL = F.sL;  // own[0] == ACT
    B.sR = tailslope;
    if (rp) { rp->b_own.clear(); rp->b_arg.clear(); }
    for (size_t q = 0; q < P.size(); ++q) {
      const int ol = own[q], orr = own[q + 1];
      const bool kink = (ol != orr) || (ol == ACT && P[q].iF >= 0);
      if (kink) {
        B.y.push_back(P[q].y); B.f.push_back(P[q].f);
        if (rp) { rp->b_own.push_back(ol); rp->b_arg.push_back(arg[q]); }
      }
    }
    if (B.y.empty()) {
      B.y.push_back(P[0].y); B.f.push_back(P[0].f);
      if (rp) { rp->b_own.push_back(own[0]); rp->b_arg.push_back(arg[0]); }
    }
    if (rp) { rp->b_own.push_back(own.back()); rp->b_arg.push_back(arg.back()); }
  }

  if (rp) {
    rp->a_y.clear();
    rp->b_y.clear();
    for (const T& y : A.y) rp->a_y.push_back(val(y));
    for (const T& y : B.y) rp->b_y.push_back(val(y));
  }
  V = pl_envelope(A, B, false, rp ? &rp->v_own : nullptr);
  return OR_OK;
}

// Expense function of the seller (Eq. 1) or of the buyer (Eq. 6):
//   seller: u(y) =  xi + (y - zeta)^- Sa - (y - zeta)^+ Sb
//   buyer : u(y) = -xi + (y + zeta)^- Sa - (y + zeta)^+ Sb
template <class T>
PL<T> pl_expense(const T& xi, const T& zeta, const T& Sa, const T& Sb, bool buyer) {
  PL<T> u;
  u.y.push_back(buyer ? -zeta : zeta);
  u.f.push_back(buyer ? -xi : xi);
  u.sL = -Sa;
  u.sR = -Sb;
  return u;
}

// One node of the induction (Section 3): w = max(z_up, z_down); f = w / r;
// v = restriction of f to slopes in [-Sa, -Sb]; z = max(u, v) (seller) or
// z = min(u, v) (buyer).
template <class T>
int node_step(const PL<T>& zu, const PL<T>& zd, const T& r, const T& Sa, const T& Sb,
              const T& xi, const T& zeta, bool buyer, PL<T>& z) {
  PL<T> w = pl_envelope(zu, zd, true);
  PL<T> f = pl_div(w, r);
  PL<T> v;
  int rc = pl_restrict(f, Sa, Sb, v);
  if (rc) return rc;
  PL<T> u = pl_expense(xi, zeta, Sa, Sb, buyer);
  z = pl_envelope(u, v, !buyer);
  return OR_OK;
}

// ---------------------------------------------------------------- derivatives by lines
// With the breakpoint structure held fixed, every piece of every function of the
// induction is a line c + s*y, and each step takes its output pieces from the lines of
// its inputs or builds new lines from them: the maximum and the minimum take the lines
// of the winning function; the division by r divides both coefficients; the flat pieces
// of the restriction are lines of slope -S^a (or -S^b) through the breakpoint y* where
// g = F + S^a y (or h = F + S^b y) attains the running minimum; the expense function is
// two lines.  So the derivatives are carried on (c, s) of every piece.  At y*, between the
// lines P (left) and Q (right) of F, the minimum value moves with
//   dg = (1 - mu) dg_P(y*) + mu dg_Q(y*),   mu = (s_P + S^a) / (s_P - s_Q),
// (y* held fixed in g_P, g_Q; at an interior minimum mu lies in [0, 1] because the slopes
// of g on the two sides bracket zero), which is the derivative of g_P(y*) with y* = the
// crossing of P and Q moving.  No breakpoint position enters a derivative: a crossing of two lines at
// a shallow angle moves fast, but the functions do not, and carrying the positions would
// cancel large terms in floating point.
struct Line {
  Dual c, s;  // value and gradient of the intercept and of the slope
};

// A function for the derivatives: its breakpoints and values (double, as priced) and
// the line of each piece: L[0] the left tail, L[k] between y[k-1] and y[k], L[m] the
// right tail.
struct LPL {
  PL<double> F;
  std::vector<Line> L;
};

// Piece of src that contains piece k of out (out's pieces lie inside src's pieces):
// the number of src breakpoints at or left of the piece's left end.
int src_piece(const std::vector<double>& src_y, const std::vector<double>& out_y, int k) {
  if (k == 0) return 0;
  return (int)(std::upper_bound(src_y.begin(), src_y.end(), out_y[k - 1]) - src_y.begin());
}

LPL lines_envelope(const LPL& X, const LPL& Y, bool take_max) {
  LPL out;
  std::vector<int> own;
  out.F = pl_envelope(X.F, Y.F, take_max, &own);
  const int m = (int)out.F.y.size();
  out.L.resize(m + 1);
  for (int k = 0; k <= m; ++k) {
    const LPL& src = (own[k] == 1) ? X : Y;
    out.L[k] = src.L[src_piece(src.F.y, out.F.y, k)];
  }
  return out;
}

LPL lines_div(const LPL& X, const Dual& r) {
  LPL out;
  out.F = pl_div(X.F, r.v);
  out.L.resize(X.L.size());
  for (size_t k = 0; k < X.L.size(); ++k) out.L[k] = Line{X.L[k].c / r, X.L[k].s / r};
  return out;
}

// Line of slope -S through the breakpoint j of F where g = F + S y is least.  Breakpoints
// that coincide with y_j to within rounding (crossings that round to within a few ulps
// of a kink) leave the choice among them to rounding noise in the values; the minimum
// sits where the slopes of the lines, + S, change sign, so j moves through such a
// cluster in the direction the lines say g keeps falling.
Line flat_line(const LPL& F, int j, const Dual& S) {
  const int m = (int)F.F.y.size();
  const double tol = 1e-12 * std::max(1.0, std::fabs(F.F.y[j]));
  while (j + 1 < m && F.L[j + 1].s.v + S.v < 0 && F.F.y[j + 1] - F.F.y[j] <= tol) ++j;
  while (j > 0 && F.L[j].s.v + S.v > 0 && F.F.y[j] - F.F.y[j - 1] <= tol) --j;
  const double ys = F.F.y[j];
  const Line& P = F.L[j];
  const Line& Q = F.L[j + 1];
  const double sp = P.s.v, sq = Q.s.v;
  const double mu = (sp == sq) ? 0.0 : (sp + S.v) / (sp - sq);
  const Dual gP = P.c + (P.s + S) * Dual(ys);
  const Dual gQ = Q.c + (Q.s + S) * Dual(ys);
  return Line{gP * Dual(1.0 - mu) + gQ * Dual(mu), -S};
}

int lines_restrict(const LPL& F, const Dual& Sa, const Dual& Sb, LPL& V) {
  RestrictPieces rp;
  int rc = pl_restrict(F.F, Sa.v, Sb.v, V.F, &rp);
  if (rc) return rc;
  enum { ACT = 1 };
  std::vector<Line> LA(rp.a_own.size()), LB(rp.b_own.size());
  for (size_t k = 0; k < LA.size(); ++k)
    LA[k] = rp.a_own[k] == ACT ? F.L[src_piece(F.F.y, rp.a_y, (int)k)] : flat_line(F, rp.a_arg[k], Sa);
  for (size_t k = 0; k < LB.size(); ++k)
    LB[k] = rp.b_own[k] == ACT ? F.L[src_piece(F.F.y, rp.b_y, (int)k)] : flat_line(F, rp.b_arg[k], Sb);
  const int m = (int)V.F.y.size();
  V.L.resize(m + 1);
  for (int k = 0; k <= m; ++k)
    V.L[k] = rp.v_own[k] == 1 ? LA[src_piece(rp.a_y, V.F.y, k)] : LB[src_piece(rp.b_y, V.F.y, k)];
  return OR_OK;
}

// Expense function (Eq. 1, Eq. 6) as two lines: left of its kink slope -S^a, right -S^b.
LPL lines_expense(const Dual& xi, const Dual& zeta, const Dual& Sa, const Dual& Sb, bool buyer) {
  LPL u;
  u.F = pl_expense<double>(xi.v, zeta.v, Sa.v, Sb.v, buyer);
  const Dual x = buyer ? -xi : xi, z = buyer ? -zeta : zeta;
  u.L = {Line{x + Sa * z, -Sa}, Line{x + Sb * z, -Sb}};  // through the kink (z, x)
  return u;
}

int lines_node_step(const LPL& zu, const LPL& zd, const Dual& r, const Dual& Sa, const Dual& Sb,
                    const Dual& xi, const Dual& zeta, bool buyer, LPL& z) {
  LPL w = lines_envelope(zu, zd, true);
  LPL f = lines_div(w, r);
  LPL v;
  int rc = lines_restrict(f, Sa, Sb, v);
  if (rc) return rc;
  LPL u = lines_expense(xi, zeta, Sa, Sb, buyer);
  z = lines_envelope(u, v, !buyer);
  return OR_OK;
}

// ---------------------------------------------------------------- tree model
template <class T>
struct Model {
  int N, payoff;
  T S0, K, K2, k, u, r;
};

int check_option(const or_option_t& o) {
  if (!(o.N >= 1) || !(o.S0 > 0) || !(o.sigma > 0) || !(o.T > 0) || !(o.k >= 0) || !(o.k < 1) ||
      !(o.K >= 0) || !std::isfinite(o.R) || o.payoff < 0 || o.payoff > 2)
    return OR_ERR_ARG;
  if (o.payoff == PAY_SPREAD && !(o.K2 >= o.K)) return OR_ERR_ARG;
  const double dt = o.T / o.N;
  const double u = std::exp(o.sigma * std::sqrt(dt));
  const double d = 1.0 / u;
  const double r = std::exp(o.R * dt);
  if (!(d < r && r < u)) return OR_ERR_ARBITRAGE;
  return OR_OK;
}

template <class T>
Model<T> make_model(const or_option_t& o, const T& S0, const T& K, const T& sigma, const T& R,
                    const T& Tm, const T& k) {
  Model<T> m;
  m.N = o.N;
  m.payoff = o.payoff;
  m.S0 = S0;
  m.K = K;
  m.K2 = T(o.K2) + (K - T(o.K));  // the spread's width is held fixed when K moves
  m.k = k;
  T dt = Tm / T((double)o.N);
  m.u = dexp(sigma * dsqrt(dt));
  m.r = dexp(R * dt);
  return m;
}

template <class T>
T stock(const Model<T>& m, int t, int j) { return m.S0 * dpowi(m.u, 2 * j - t); }

template <class T>
void payoff_at(const Model<T>& m, const T& S, T& xi, T& zeta) {
  if (m.payoff == PAY_PUT) { xi = m.K; zeta = T(-1.0); }
  else if (m.payoff == PAY_CALL) { xi = -m.K; zeta = T(1.0); }
  else {
    T a = (val(S) > val(m.K)) ? S - m.K : T(0.0);
    T b = (val(S) > val(m.K2)) ? S - m.K2 : T(0.0);
    xi = a - b;
    zeta = T(0.0);
  }
}

struct Stats {
  int64_t nodes = 0;
  int64_t bp_seller = 0, bp_buyer = 0;   // sum of breakpoints over all computed nodes
  int max_seller = 0, max_buyer = 0;
  std::vector<int64_t>* per_level = nullptr;  // optional: [2*(N+2)] sums by level
};

// z1 (may be null) receives level 1's functions: seller j = 0, 1, then buyer j = 0, 1.
template <class T>
int price_tc(const Model<T>& m, T& ask, T& bid, Stats* st, PL<T>* z1 = nullptr) {
  const int N = m.N;
  std::vector<PL<T>> zs(N + 2), zb(N + 2);
  // level N+1: payoff (0, 0) for both parties; costs apply there.
  for (int j = 0; j <= N + 1; ++j) {
    T S = stock(m, N + 1, j);
    T Sa = (T(1.0) + m.k) * S, Sb = (T(1.0) - m.k) * S;
    zs[j] = pl_expense(T(0.0), T(0.0), Sa, Sb, false);
    zb[j] = pl_expense(T(0.0), T(0.0), Sa, Sb, true);
  }
  for (int t = N; t >= 0; --t) {
    for (int j = 0; j <= t; ++j) {  // ascending j: slot j+1 still holds level t+1
      T S = stock(m, t, j);
      T kt = (t == 0) ? T(0.0) : m.k;
      T Sa = (T(1.0) + kt) * S, Sb = (T(1.0) - kt) * S;
      T xi, zeta;
      payoff_at(m, S, xi, zeta);
      PL<T> ns, nb;
      int rc = node_step(zs[j + 1], zs[j], m.r, Sa, Sb, xi, zeta, false, ns);
      if (rc) return rc;
      rc = node_step(zb[j + 1], zb[j], m.r, Sa, Sb, xi, zeta, true, nb);
      if (rc) return rc;
      zs[j] = std::move(ns);
      zb[j] = std::move(nb);
      if (st) {
        st->nodes += 1;
        const int ms = (int)zs[j].y.size(), mb = (int)zb[j].y.size();
        st->bp_seller += ms;
        st->bp_buyer += mb;
        st->max_seller = std::max(st->max_seller, ms);
        st->max_buyer = std::max(st->max_buyer, mb);
        if (st->per_level) {
          (*st->per_level)[2 * t] += ms;
          (*st->per_level)[2 * t + 1] += mb;
        }
      }
    }
    if (t == 1 && z1) {
      z1[0] = zs[0]; z1[1] = zs[1];
      z1[2] = zb[0]; z1[3] = zb[1];
    }
  }
  ask = pl_eval(zs[0], T(0.0));
  bid = -pl_eval(zb[0], T(0.0));
  return OR_OK;
}

// The induction of price_tc on LPL functions: the same prices (the breakpoints and values
// are computed by the same double functions), and their derivatives through the lines.
// The value at y = 0 of the root functions is that of the piece right of every breakpoint
// at or left of 0.
int price_tc_lines(const Model<Dual>& m, Dual& ask, Dual& bid) {
  const int N = m.N;
  std::vector<LPL> zs(N + 2), zb(N + 2);
  for (int j = 0; j <= N + 1; ++j) {
    Dual S = stock(m, N + 1, j);
    Dual Sa = (Dual(1.0) + m.k) * S, Sb = (Dual(1.0) - m.k) * S;
    zs[j] = lines_expense(Dual(0.0), Dual(0.0), Sa, Sb, false);
    zb[j] = lines_expense(Dual(0.0), Dual(0.0), Sa, Sb, true);
  }
  for (int t = N; t >= 0; --t) {
    for (int j = 0; j <= t; ++j) {
      Dual S = stock(m, t, j);
      Dual kt = (t == 0) ? Dual(0.0) : m.k;
      Dual Sa = (Dual(1.0) + kt) * S, Sb = (Dual(1.0) - kt) * S;
      Dual xi, zeta;
      payoff_at(m, S, xi, zeta);
      LPL ns, nb;
      int rc = lines_node_step(zs[j + 1], zs[j], m.r, Sa, Sb, xi, zeta, false, ns);
      if (rc) return rc;
      rc = lines_node_step(zb[j + 1], zb[j], m.r, Sa, Sb, xi, zeta, true, nb);
      if (rc) return rc;
      zs[j] = std::move(ns);
      zb[j] = std::move(nb);
    }
  }
  auto at0 = [](const LPL& z) {
    const int k = (int)(std::upper_bound(z.F.y.begin(), z.F.y.end(), 0.0) - z.F.y.begin());
    Dual v = z.L[k].c;  // c + s * 0
    v.v = pl_eval(z.F, 0.0);
    return v;
  };
  ask = at0(zs[0]);
  bid = -at0(zb[0]);
  return OR_OK;
}

// Plain CRR recursion without costs (Section 3, Appendix): N levels, no extra
// level; exercise value P_t = K - S (put), S - K (call), spread payoff.
double crr_payoff(int payoff, double S, double K, double K2) {
  if (payoff == PAY_PUT) return K - S;
  if (payoff == PAY_CALL) return S - K;
  return std::max(S - K, 0.0) - std::max(S - K2, 0.0);
}

double price_crr(const or_option_t& o, bool american) {
  const int N = o.N;
  const double dt = o.T / N;
  const double u = std::exp(o.sigma * std::sqrt(dt));
  const double d = 1.0 / u;
  const double r = std::exp(o.R * dt);
  const double p = (r - d) / (u - d);
  std::vector<double> c(N + 1);
  for (int j = 0; j <= N; ++j)
    c[j] = std::max(crr_payoff(o.payoff, o.S0 * std::pow(u, 2 * j - N), o.K, o.K2), 0.0);
  for (int t = N - 1; t >= 0; --t) {
    for (int j = 0; j <= t; ++j) {
      const double cont = (p * c[j + 1] + (1.0 - p) * c[j]) / r;
      c[j] = american ? std::max(crr_payoff(o.payoff, o.S0 * std::pow(u, 2 * j - t), o.K, o.K2), cont)
                      : cont;
    }
  }
  return c[0];
}

template <class F>
void parallel_for(int64_t n, int nthreads, F fn) {
  if (nthreads <= 1 || n <= 1) {
    for (int64_t i = 0; i < n; ++i) fn(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> pool;
  for (int w = 0; w < nthreads; ++w)
    pool.emplace_back([&]() {
      for (;;) {
        int64_t i = next.fetch_add(1);
        if (i >= n) break;
        fn(i);
      }
    });
  for (auto& th : pool) th.join();
}

template <class T>
PL<T> pl_from(const double* y, const double* f, int m, double sL, double sR) {
  PL<T> F;
  for (int i = 0; i < m; ++i) { F.y.push_back(T(y[i])); F.f.push_back(T(f[i])); }
  F.sL = T(sL);
  F.sR = T(sR);
  return F;
}

int pl_to(const PL<double>& F, double* y, double* f, int cap, double* sL, double* sR) {
  const int m = (int)F.y.size();
  if (m > cap) return OR_ERR_CAPACITY;
  for (int i = 0; i < m; ++i) { y[i] = F.y[i]; f[i] = F.f[i]; }
  *sL = F.sL;
  *sR = F.sR;
  return m;
}

// ---------------------------------------------------------------- the initial hedge
// Section 3: a portfolio (x, y) at time t covers the seller from t+1 on iff, after
// rebalancing the stock holding from y to some y' (buying at S^a, selling at S^b), the
// cash left lies above w_t/r at y'; v_t(y) = inf_{y'} [F(y') + theta(y' - y)], F = w_t/r.
// The y' that attains it is the holding the hedger moves to.  F + theta(. - y) is piecewise
// linear with kinks at F's breakpoints and at y, so the infimum is attained at one of them
// (the tails rise away from them when the restriction is bounded).  Among equal minima the
// rightmost is taken.  Returns OR_ERR_UNBOUNDED when a tail falls.
template <class T>
int pl_rebalance(const PL<T>& F, double Sa, double Sb, double y, double& yopt, double& vopt) {
  if (val(F.sR) + Sa < 0 || val(F.sL) + Sb > 0) return OR_ERR_UNBOUNDED;
  std::vector<double> cand;
  for (const T& b : F.y) cand.push_back(val(b));
  cand.push_back(y);
  std::sort(cand.begin(), cand.end());
  bool have = false;
  for (double c : cand) {
    const double v = val(pl_eval(F, T(c))) + (c >= y ? Sa : Sb) * (c - y);
    if (!have || v <= vopt) {
      vopt = v;
      yopt = c;
      have = true;
    }
  }
  return OR_OK;
}

// The hedge at the root: for the seller (p = 0) and the buyer (p = 1), the stock holding y*
// that a hedger starting from no stock moves to at t = 0 (no costs there: theta(x) = S0 x),
// v_0(0) = F(y*) + S0 y*, and whether immediate exercise sets the price (seller:
// u_0(0) > v_0(0)) or is the buyer's choice (u_0(0) < v_0(0)).
int initial_hedge(const Model<double>& m, double* out) {
  PL<double> z1[4];
  double ask, bid;
  int rc = price_tc(m, ask, bid, nullptr, z1);
  if (rc) return rc;
  double xi, zeta;
  payoff_at(m, m.S0, xi, zeta);
  for (int p = 0; p < 2; ++p) {
    PL<double> w = pl_envelope(z1[2 * p + 1], z1[2 * p], true);  // up successor j = 1
    PL<double> f = pl_div(w, m.r);
    double ys = 0.0, vs = 0.0;
    rc = pl_rebalance(f, m.S0, m.S0, 0.0, ys, vs);
    if (rc) return rc;
    const double u0 = pl_eval(pl_expense(xi, zeta, m.S0, m.S0, p == 1), 0.0);
    out[p] = ys;
    out[2 + p] = (p == 0) ? (u0 > vs ? 1.0 : 0.0) : (u0 < vs ? 1.0 : 0.0);
  }
  return OR_OK;
}

// The hedge along one path of the tree: the same rebalancing at every node the path visits.
// moves[t] = 1 for an up move from level t to t+1, 0 for a down move (t < N); the path's node
// at level t is j_t = the number of up moves before t.  hold[2t] is the seller's stock holding
// after rebalancing at t (from the previous holding, 0 before t = 0; to the y' attaining
// v_t(y) = inf_y' [w_t(y')/r + theta_t(y' - y)]), hold[2t+1] the buyer's; the buyer stops at the
// first t where u_t(y) < v_t(y) for the holding y it arrives with (*stop = t, NaN from there
// on; -1 if it never does).  The functions w_t of the path's nodes are kept during the
// induction of price_tc (built the same way).  cash[2t] and cash[2t+1] are the parties' cash
// after rebalancing at t, in time-t money, of the self-financing portfolios that start at
// t = 0 with no stock and the ask (seller) or minus the bid (buyer, who borrows it to buy the
// option): x_t = r x_{t-1} - theta_t(y_t - y_{t-1}), x_{-1} r = ask or -bid.
int hedge_path(const Model<double>& m, const int8_t* moves, double* hold, double* cash, int* stop) {
  const int N = m.N;
  std::vector<int> jt(N + 1, 0);
  for (int t = 1; t <= N; ++t) jt[t] = jt[t - 1] + (moves[t - 1] ? 1 : 0);
  std::vector<PL<double>> zs(N + 2), zb(N + 2), Fs(N + 1), Fb(N + 1);
  for (int j = 0; j <= N + 1; ++j) {
    const double S = stock(m, N + 1, j);
    const double Sa = (1.0 + m.k) * S, Sb = (1.0 - m.k) * S;
    zs[j] = pl_expense(0.0, 0.0, Sa, Sb, false);
    zb[j] = pl_expense(0.0, 0.0, Sa, Sb, true);
  }
  for (int t = N; t >= 0; --t) {
    for (int j = 0; j <= t; ++j) {
      const double S = stock(m, t, j);
      const double kt = (t == 0) ? 0.0 : m.k;
      const double Sa = (1.0 + kt) * S, Sb = (1.0 - kt) * S;
      double xi, zeta;
      payoff_at(m, S, xi, zeta);
      if (j == jt[t]) {  // the path's node: keep w / r
        Fs[t] = pl_div(pl_envelope(zs[j + 1], zs[j], true), m.r);
        Fb[t] = pl_div(pl_envelope(zb[j + 1], zb[j], true), m.r);
      }
      PL<double> ns, nb;
      int rc = node_step(zs[j + 1], zs[j], m.r, Sa, Sb, xi, zeta, false, ns);
      if (rc) return rc;
      rc = node_step(zb[j + 1], zb[j], m.r, Sa, Sb, xi, zeta, true, nb);
      if (rc) return rc;
      zs[j] = std::move(ns);
      zb[j] = std::move(nb);
    }
  }
  double ys = 0.0, yb = 0.0;
  double xs = pl_eval(zs[0], 0.0), xb = pl_eval(zb[0], 0.0);  // ask and -bid
  *stop = -1;
  for (int t = 0; t <= N; ++t) {
    const double S = stock(m, t, jt[t]);
    const double kt = (t == 0) ? 0.0 : m.k;
    const double Sa = (1.0 + kt) * S, Sb = (1.0 - kt) * S;
    double y = 0.0, v = 0.0;
    int rc = pl_rebalance(Fs[t], Sa, Sb, ys, y, v);
    if (rc) return rc;
    if (t > 0) xs *= m.r;
    xs -= (y >= ys ? Sa : Sb) * (y - ys);
    hold[2 * t] = ys = y;
    cash[2 * t] = xs;
    if (*stop >= 0) {
      hold[2 * t + 1] = NAN;
      cash[2 * t + 1] = NAN;
      continue;
    }
    if ((rc = pl_rebalance(Fb[t], Sa, Sb, yb, y, v))) return rc;
    double xi, zeta;
    payoff_at(m, S, xi, zeta);
    const double u = pl_eval(pl_expense(xi, zeta, Sa, Sb, true), yb);
    if (u < v) {
      *stop = t;
      hold[2 * t + 1] = NAN;
      cash[2 * t + 1] = NAN;
    } else {
      if (t > 0) xb *= m.r;
      xb -= (y >= yb ? Sa : Sb) * (y - yb);
      hold[2 * t + 1] = yb = y;
      cash[2 * t + 1] = xb;
    }
  }
  return OR_OK;
}

// ---------------------------------------------------------------- Algorithm 1 (Section 4.2)
// The paper's parallel scheme for one option on p threads, driving the node steps above
// (price_tc's and price_crr's arithmetic, node for node, so the results are bitwise the
// serial ones).  The tree is processed in rounds.  A round starts at a base level B whose
// B+1 nodes were finished in the previous round; it computes the levels B-1 .. B-D.
//   * Threads: while B+1 < 2p, p drops by one (every thread gets at least two nodes), so a
//     retired thread takes no further part.
//   * Blocks: thread i takes the columns [i q, (i+1) q) of every level of the round,
//     q = floor((B+1)/p); the last thread takes the rest.  D = min(L, q - 1) >= 1.
//   * Regions: the nodes of a block at level B-o whose two successors lie in the block's
//     columns, [s, e-o), form region A (no dependence on other threads).  The remaining
//     columns [e-o, e) form region B: node (B-o, e-1) needs column e = the next thread's
//     first column at level B-o+1.
//   * Synchronisation: thread i > 0 signals thread i-1 once it has finished the node of its
//     first column at level B-D+1 (B-1 when D = 1); region A goes level by level, so by
//     then every node of that column that thread i-1 reads is done.  Thread i-1 computes its
//     region B after its region A and that signal.  All active threads meet at a barrier at
//     the end of the round.
//   * Storage: (L+1) rows of N+2 cells per party; level t lives in row t mod (L+1) (a round
//     touches D+1 <= L+1 consecutive levels, so no two of them share a row).
// Reading: the paper's listing uses n for a base level's index in one place and for its
// node count in another, and gives the last block's size two ways; the node count B+1 and
// the contiguous split above are taken.

struct Alg1Round {
  int B, D, p;
};

std::vector<Alg1Round> alg1_rounds(int top, int p, int L) {
  std::vector<Alg1Round> r;
  if (p < 1) p = 1;
  if (L < 1) L = 1;
  for (int B = top; B > 0;) {
    while (p > 1 && B + 1 < 2 * p) --p;
    const int q = (B + 1) / p;
    const int D = std::min(L, q - 1);
    r.push_back({B, D, p});
    B -= D;
  }
  return r;
}

// A barrier for the threads of one round (their count is the same for all of them).
struct RoundBarrier {
  std::mutex mu;
  std::condition_variable cv;
  int arrived = 0;
  int64_t gen = 0;
  void arrive(int count) {
    std::unique_lock<std::mutex> lk(mu);
    const int64_t g = gen;
    if (++arrived == count) {
      arrived = 0;
      ++gen;
      cv.notify_all();
    } else {
      cv.wait(lk, [&] { return gen != g; });
    }
  }
};

// Runs the rounds on p threads.  node(t, j) computes node (t, j) from level t+1 and returns
// an error code (0 = OK); init(j) sets leaf j of level top.  nodes_per_thread (may be null)
// receives the number of nodes each thread computed.
template <class Node, class Init>
int alg1_run(int top, int p, int L, Node node, Init init, int64_t* nodes_per_thread) {
  const std::vector<Alg1Round> rounds = alg1_rounds(top, p, L);
  if (p < 1) p = 1;
  if (L < 1) L = 1;
  std::vector<std::atomic<int>> sig(p);
  for (auto& g : sig) g.store(0);
  std::atomic<int> err(0);
  RoundBarrier bar;
  std::vector<int64_t> count(p, 0);
  auto body = [&](int i) {
    int64_t done = 0;  // nodes computed by this thread (kept local: no shared cache line)
    {  // leaves, split as in the first round
      const int P0 = rounds.empty() ? 1 : rounds[0].p;
      if (i >= P0) return;
      const int n = top + 1, q = n / P0;
      const int s = i * q, e = (i == P0 - 1) ? n : (i + 1) * q;
      for (int j = s; j < e; ++j) init(j);
      bar.arrive(P0);
    }
    for (size_t k = 0; k < rounds.size(); ++k) {
      const Alg1Round& R = rounds[k];
      if (i >= R.p) break;
      const int n = R.B + 1, q = n / R.p;
      const int s = i * q, e = (i == R.p - 1) ? n : (i + 1) * q;
      const int sig_level = (R.D > 1) ? R.B - R.D + 1 : R.B - 1;
      auto compute = [&](int t, int j) {
        if (err.load(std::memory_order_relaxed)) return;
        const int rc = node(t, j);
        if (rc) err.store(rc);
        ++done;
      };
      for (int o = 1; o <= R.D; ++o) {  // region A, level by level
        const int t = R.B - o;
        const int m = std::min(e - o, t + 1);
        for (int j = s; j < m; ++j) {
          compute(t, j);
          if (i > 0 && t == sig_level && j == s) sig[i].store((int)k + 1, std::memory_order_release);
        }
      }
      if (i + 1 < R.p) {  // region B, after the next thread's signal
        while (sig[i + 1].load(std::memory_order_acquire) < (int)k + 1) std::this_thread::yield();
        for (int o = 1; o <= R.D; ++o) {
          const int t = R.B - o;
          for (int j = std::max(s, e - o); j < e && j <= t; ++j) compute(t, j);
        }
      }
      bar.arrive(R.p);
    }
    count[i] = done;
  };
  std::vector<std::thread> pool;
  for (int i = 1; i < p; ++i) pool.emplace_back(body, i);
  body(0);
  for (auto& th : pool) th.join();
  if (nodes_per_thread)
    for (int i = 0; i < p; ++i) nodes_per_thread[i] = count[i];
  return err.load();
}

// ask and bid of one option (the model of price_tc) by Algorithm 1.
int alg1_tc(const or_option_t& o, int p, int L, double& ask, double& bid, int64_t* per_thread) {
  const Model<double> m = make_model<double>(o, o.S0, o.K, o.sigma, o.R, o.T, o.k);
  const int N = m.N, rows = std::max(L, 1) + 1;
  std::vector<PL<double>> zs((size_t)rows * (N + 2)), zb((size_t)rows * (N + 2));
  auto cell = [&](std::vector<PL<double>>& z, int t, int j) -> PL<double>& {
    return z[(size_t)(t % rows) * (N + 2) + j];
  };
  auto init = [&](int j) {
    const double S = stock(m, N + 1, j);
    const double Sa = (1.0 + m.k) * S, Sb = (1.0 - m.k) * S;
    cell(zs, N + 1, j) = pl_expense(0.0, 0.0, Sa, Sb, false);
    cell(zb, N + 1, j) = pl_expense(0.0, 0.0, Sa, Sb, true);
  };
  auto node = [&](int t, int j) -> int {
    const double S = stock(m, t, j);
    const double kt = (t == 0) ? 0.0 : m.k;
    const double Sa = (1.0 + kt) * S, Sb = (1.0 - kt) * S;
    double xi, zeta;
    payoff_at(m, S, xi, zeta);
    int rc = node_step(cell(zs, t + 1, j + 1), cell(zs, t + 1, j), m.r, Sa, Sb, xi, zeta, false,
                       cell(zs, t, j));
    if (rc) return rc;
    return node_step(cell(zb, t + 1, j + 1), cell(zb, t + 1, j), m.r, Sa, Sb, xi, zeta, true,
                     cell(zb, t, j));
  };
  const int rc = alg1_run(N + 1, p, L, node, init, per_thread);
  if (rc) return rc;
  ask = pl_eval(cell(zs, 0, 0), 0.0);
  bid = -pl_eval(cell(zb, 0, 0), 0.0);
  return OR_OK;
}

// The American CRR price (the recursion of price_crr) by Algorithm 1.
int alg1_crr(const or_option_t& o, int p, int L, double& price, int64_t* per_thread) {
  const int N = o.N, rows = std::max(L, 1) + 1;
  const double dt = o.T / N;
  const double u = std::exp(o.sigma * std::sqrt(dt));
  const double d = 1.0 / u;
  const double r = std::exp(o.R * dt);
  const double pu = (r - d) / (u - d);
  std::vector<double> c((size_t)rows * (N + 1));
  auto cell = [&](int t, int j) -> double& { return c[(size_t)(t % rows) * (N + 1) + j]; };
  auto init = [&](int j) {
    cell(N, j) = std::max(crr_payoff(o.payoff, o.S0 * std::pow(u, 2 * j - N), o.K, o.K2), 0.0);
  };
  auto node = [&](int t, int j) -> int {
    const double cont = (pu * cell(t + 1, j + 1) + (1.0 - pu) * cell(t + 1, j)) / r;
    cell(t, j) = std::max(crr_payoff(o.payoff, o.S0 * std::pow(u, 2 * j - t), o.K, o.K2), cont);
    return OR_OK;
  };
  const int rc = alg1_run(N, p, L, node, init, per_thread);
  if (rc) return rc;
  price = cell(0, 0);
  return OR_OK;
}

}  // namespace

extern "C" {

// ask/bid of each option by the piecewise-linear induction; out[2i] = ask,
// out[2i+1] = bid; status[i] = 0 or a negative error code.
int or_price_tc(const or_option_t* opts, int64_t n, double* out, int32_t* status, int nthreads) {
  parallel_for(n, nthreads, [&](int64_t i) {
    const or_option_t& o = opts[i];
    int rc = check_option(o);
    double ask = NAN, bid = NAN;
    if (rc == OR_OK) {
      Model<double> m = make_model<double>(o, o.S0, o.K, o.sigma, o.R, o.T, o.k);
      rc = price_tc(m, ask, bid, nullptr);
    }
    out[2 * i] = ask;
    out[2 * i + 1] = bid;
    if (status) status[i] = rc;
  });
  return OR_OK;
}

// Breakpoint statistics of one option's induction: counts[0] = nodes,
// [1] = sum of seller breakpoints, [2] = sum of buyer breakpoints,
// [3] = max seller, [4] = max buyer.  per_level (may be NULL) receives
// 2*(N+1) sums: [2t] seller, [2t+1] buyer, for t = 0..N.
int or_tc_stats(const or_option_t* o, int64_t* counts, int64_t* per_level) {
  int rc = check_option(*o);
  if (rc) return rc;
  Model<double> m = make_model<double>(*o, o->S0, o->K, o->sigma, o->R, o->T, o->k);
  Stats st;
  std::vector<int64_t> pl(2 * (o->N + 1), 0);
  st.per_level = &pl;
  double ask, bid;
  rc = price_tc(m, ask, bid, &st);
  if (rc) return rc;
  counts[0] = st.nodes;
  counts[1] = st.bp_seller;
  counts[2] = st.bp_buyer;
  counts[3] = st.max_seller;
  counts[4] = st.max_buyer;
  if (per_level) std::memcpy(per_level, pl.data(), pl.size() * sizeof(int64_t));
  return OR_OK;
}

// Derivatives of ask and bid by forward-mode dual numbers carried on the lines of the
// pieces (price_tc_lines): grad[12i + 0..5] = d ask / d(S0, K, sigma, R, T, k),
// grad[12i + 6..11] = d bid / d(...).
int or_greeks_tc(const or_option_t* opts, int64_t n, double* out, double* grad, int32_t* status,
                 int nthreads) {
  parallel_for(n, nthreads, [&](int64_t i) {
    const or_option_t& o = opts[i];
    int rc = check_option(o);
    Dual ask, bid;
    if (rc == OR_OK) {
      Dual in[NG];
      const double base[NG] = {o.S0, o.K, o.sigma, o.R, o.T, o.k};
      for (int a = 0; a < NG; ++a) { in[a] = Dual(base[a]); in[a].g[a] = 1.0; }
      Model<Dual> m = make_model<Dual>(o, in[0], in[1], in[2], in[3], in[4], in[5]);
      rc = price_tc_lines(m, ask, bid);
    }
    out[2 * i] = rc ? NAN : ask.v;
    out[2 * i + 1] = rc ? NAN : bid.v;
    for (int a = 0; a < NG; ++a) {
      grad[12 * i + a] = rc ? NAN : ask.g[a];
      grad[12 * i + 6 + a] = rc ? NAN : bid.g[a];
    }
    if (status) status[i] = rc;
  });
  return OR_OK;
}

// Plain CRR price without costs; american = 0 gives the European price.
int or_price_crr(const or_option_t* opts, int64_t n, double* out, int32_t* status, int american,
                 int nthreads) {
  parallel_for(n, nthreads, [&](int64_t i) {
    int rc = check_option(opts[i]);
    out[i] = rc ? NAN : price_crr(opts[i], american != 0);
    if (status) status[i] = rc;
  });
  return OR_OK;
}

// ---- single primitives on explicit PL functions (for unit tests) ----
int or_pl_envelope(const double* y1, const double* f1, int m1, double sL1, double sR1,
                   const double* y2, const double* f2, int m2, double sL2, double sR2, int take_max,
                   double* yo, double* fo, int cap, double* sLo, double* sRo) {
  if (m1 < 1 || m2 < 1) return OR_ERR_ARG;
  PL<double> F = pl_from<double>(y1, f1, m1, sL1, sR1), G = pl_from<double>(y2, f2, m2, sL2, sR2);
  return pl_to(pl_envelope(F, G, take_max != 0), yo, fo, cap, sLo, sRo);
}

int or_pl_restrict(const double* y, const double* f, int m, double sL, double sR, double Sa,
                   double Sb, double* yo, double* fo, int cap, double* sLo, double* sRo) {
  if (m < 1) return OR_ERR_ARG;
  PL<double> F = pl_from<double>(y, f, m, sL, sR), V;
  int rc = pl_restrict(F, Sa, Sb, V);
  if (rc) return rc;
  return pl_to(V, yo, fo, cap, sLo, sRo);
}

int or_pl_eval(const double* y, const double* f, int m, double sL, double sR, const double* x,
               int nx, double* out) {
  if (m < 1) return OR_ERR_ARG;
  PL<double> F = pl_from<double>(y, f, m, sL, sR);
  for (int i = 0; i < nx; ++i) out[i] = pl_eval(F, x[i]);
  return OR_OK;
}

// One node of the induction from explicit successor functions.
int or_node_step(const double* yu, const double* fu, int mu, double sLu, double sRu,
                 const double* yd, const double* fd, int md, double sLd, double sRd, double r,
                 double Sa, double Sb, double xi, double zeta, int buyer, double* yo, double* fo,
                 int cap, double* sLo, double* sRo) {
  if (mu < 1 || md < 1) return OR_ERR_ARG;
  PL<double> U = pl_from<double>(yu, fu, mu, sLu, sRu), D = pl_from<double>(yd, fd, md, sLd, sRd);
  PL<double> z;
  int rc = node_step(U, D, r, Sa, Sb, xi, zeta, buyer != 0, z);
  if (rc) return rc;
  return pl_to(z, yo, fo, cap, sLo, sRo);
}


// ---- Algorithm 1 (Section 4.2) on p threads with blocks of at most L levels ----
// One option; out[0] = ask, out[1] = bid (or_alg1_tc) or out[0] = the American CRR price
// (or_alg1_crr); per_thread (may be NULL) receives the nodes each of the p threads computed.
// Returns 0 or an error code (also in *status).
int or_alg1_tc(const or_option_t* o, int p, int L, double* out, int32_t* status,
               int64_t* per_thread) {
  int rc = check_option(*o);
  double ask = NAN, bid = NAN;
  if (rc == OR_OK) rc = alg1_tc(*o, p, L, ask, bid, per_thread);
  out[0] = rc ? NAN : ask;
  out[1] = rc ? NAN : bid;
  if (status) *status = rc;
  return rc;
}

int or_alg1_crr(const or_option_t* o, int p, int L, double* out, int32_t* status,
                int64_t* per_thread) {
  int rc = check_option(*o);
  double c = NAN;
  if (rc == OR_OK) rc = alg1_crr(*o, p, L, c, per_thread);
  out[0] = rc ? NAN : c;
  if (status) *status = rc;
  return rc;
}

// The rounds of Algorithm 1 from base level `top`: (B, D, p) per round into out (3 ints a
// round, at most cap rounds).  Returns the number of rounds.
int or_alg1_rounds(int top, int p, int L, int32_t* out, int cap) {
  const std::vector<Alg1Round> r = alg1_rounds(top, p, L);
  for (size_t k = 0; k < r.size() && (int)k < cap; ++k) {
    out[3 * k] = r[k].B;
    out[3 * k + 1] = r[k].D;
    out[3 * k + 2] = r[k].p;
  }
  return (int)r.size();
}


// The hedge at the root of each option (initial_hedge): out[4i] = the seller's stock
// holding after rebalancing at t = 0, out[4i+1] the buyer's, out[4i+2] = 1 when immediate
// exercise sets the ask, out[4i+3] = 1 when the buyer exercises at once.
int or_initial_hedge(const or_option_t* opts, int64_t n, double* out, int32_t* status, int nthreads) {
  parallel_for(n, nthreads, [&](int64_t i) {
    const or_option_t& o = opts[i];
    int rc = check_option(o);
    if (rc == OR_OK) {
      Model<double> m = make_model<double>(o, o.S0, o.K, o.sigma, o.R, o.T, o.k);
      rc = initial_hedge(m, out + 4 * i);
    }
    if (rc)
      for (int c = 0; c < 4; ++c) out[4 * i + c] = NAN;
    if (status) status[i] = rc;
  });
  return OR_OK;
}

// The objective of the root's rebalancing, F(y) + S0 y with F = w_0/r of party p (0 seller,
// 1 buyer), at ny holdings y (for checking a hedge that another minimiser of equal value
// chose).
int or_root_objective(const or_option_t* o, int p, const double* y, int ny, double* out) {
  int rc = check_option(*o);
  if (rc) return rc;
  Model<double> m = make_model<double>(*o, o->S0, o->K, o->sigma, o->R, o->T, o->k);
  PL<double> z1[4];
  double ask, bid;
  if ((rc = price_tc(m, ask, bid, nullptr, z1))) return rc;
  const PL<double> f = pl_div(pl_envelope(z1[2 * p + 1], z1[2 * p], true), m.r);
  for (int i = 0; i < ny; ++i) out[i] = pl_eval(f, y[i]) + m.S0 * y[i];
  return OR_OK;
}

// The rebalancing target of pl_rebalance on an explicit PL function (for unit tests).
int or_pl_rebalance(const double* y, const double* f, int m, double sL, double sR, double Sa,
                    double Sb, double y0, double* yopt, double* vopt) {
  if (m < 1) return OR_ERR_ARG;
  PL<double> F = pl_from<double>(y, f, m, sL, sR);
  return pl_rebalance(F, Sa, Sb, y0, *yopt, *vopt);
}


// The hedge along a path for each option (hedge_path): moves + i * stride holds option i's N
// moves, hold + 2 * (stride + 1) * i its 2 (N + 1) holdings, cash (same layout) the parties'
// cash after rebalancing, stop[i] the buyer's stopping time.
int or_hedge_path(const or_option_t* opts, int64_t n, const int8_t* moves, int64_t stride,
                  double* hold, double* cash, int32_t* stop, int32_t* status, int nthreads) {
  parallel_for(n, nthreads, [&](int64_t i) {
    const or_option_t& o = opts[i];
    double* h = hold + 2 * (stride + 1) * i;
    double* c = cash + 2 * (stride + 1) * i;
    int rc = check_option(o);
    if (rc == OR_OK && o.N > stride) rc = OR_ERR_ARG;
    int st = -1;
    if (rc == OR_OK) {
      Model<double> m = make_model<double>(o, o.S0, o.K, o.sigma, o.R, o.T, o.k);
      rc = hedge_path(m, moves + stride * i, h, c, &st);
    }
    for (int64_t k = rc ? 0 : 2 * ((int64_t)o.N + 1); k < 2 * (stride + 1); ++k) h[k] = c[k] = NAN;
    stop[i] = rc ? -1 : st;
    if (status) status[i] = rc;
  });
  return OR_OK;
}

}  // extern "C"
