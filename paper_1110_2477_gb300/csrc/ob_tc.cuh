// ob_tc.cuh -- the level-by-level backward induction of the seller's (ask) and
// buyer's (bid) piecewise-linear functions on a recombining binomial tree
// (Zhang, Roux & Zastawniak, Section 3 and Section 4.1; the sequential
// procedures are Roux & Zastawniak's Algorithms 3.1 and 3.5), written as
// element-parallel passes for one team of threads (a warp or a whole CTA) working
// on one option; TcGroup at the end splits each level over several teams.
//
// Representation.  A node function is a list of breakpoints (y, value,
// slope to the right of y).  Its left-tail slope is always -S^a_t and its
// right-tail slope -S^b_t (both children's tails bracket the window whenever
// d < r < u, so the restriction clips them), so tails are not stored.
// Values are kept in "future-value" units: a value at level t is multiplied by
// lambda_t = r^(N+1-t).  Discounting w_t by r then costs nothing, and a slope
// is never rescaled once created, so two pieces with the same origin keep
// bitwise-equal slopes and a breakpoint between them can be dropped exactly.
//
// One level t (from level t+1):
//   pass 1  for each breakpoint of the two successors (a merge of their sorted
//           lists): evaluate both successors there, keep w = max(z_up, z_down),
//           insert the crossings between neighbouring points and in the tails.
//   pass 2  g = w + S^a y and h = w + S^b y at every point of w, then the
//           running minima cA (suffix, from the right) and cB (prefix, from the
//           left) per node, as segmented scans on integer keys.
//   pass 3  for every piece of w: the restriction
//             v = min( w-line, cA_{i+1} - S^a y, cB_i - S^b y )
//           (the inf-convolution v(y) = inf_y' [w(y') + theta(y' - y)] split into
//           buying and selling; on the left tail v is the cA line, on the right
//           tail the cB line), then z = max(u, v) for the seller or
//           z = min(u, v) for the buyer, with u the expense function (Eq. 1,
//           Eq. 6).  A point is emitted only where the slope changes.
#pragma once
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "ob_team.cuh"

namespace obk {

enum { ST_OK = 0, ST_ARG = -1, ST_ARBITRAGE = -2, ST_CAPACITY = -3 };
enum { PAY_PUT = 0, PAY_CALL = 1, PAY_SPREAD = 2 };

struct Opt {
  double S0, K, K2, sigma, R, T, k;
  int32_t N, payoff;
};

struct Stats {
  long long upts;        // successor breakpoints merged (union points) over all levels
  long long wpts, zpts;  // points of w and of z summed over all levels (both parties)
  int zmax_level;        // largest number of z points in one level
  double hedge[4];       // the hedge at the root (TcRun::root_hedge)
};

// Per-option scratch carved from one worker's arena.
struct Lay {
  double* Stab;   // [2N+3]   S0 u^e, e = -(N+1)..N+1 at index e+N+1
  double* lam;    // [N+2]    lambda_t = r^(N+1-t)
  double* nt[2];  // [4(N+2)] per node of a level: S^a lambda, S^b lambda, xi lambda
  int* off[2];    // [2(N+2)+1] first point of each node (seller nodes, then buyer nodes)
  double *zY[2], *zF[2], *zS[2];
  int* wN;        // node of each point of w
  double *wY, *wF, *wS;
  long long *wGK, *wHK;  // keys of g = w + S^a y and h = w + S^b y (only compared)
  long long *wCA, *wCB;
  int capZ, capW;
};

OB_HD size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes of the per-option node arrays for N steps.
OB_HD size_t node_bytes(int N) {
  size_t n = 0;
  n += al256(sizeof(double) * (2 * (size_t)N + 3));
  n += al256(sizeof(double) * ((size_t)N + 2));
  n += 2 * al256(sizeof(double) * 4 * ((size_t)N + 2));
  n += 2 * al256(sizeof(int) * (2 * ((size_t)N + 2) + 1));
  return n;
}

constexpr size_t ELEM_BYTES = 2 * 3 * sizeof(double) + 5 * sizeof(double) + 2 * sizeof(long long) +
                              sizeof(int);

// Carve the arrays for N steps and `cap` points per array starting at base;
// returns the first byte after them.
OB_HD char* carve_cap(char* base, int N, size_t cap, Lay& L) {
  char* p = base;
  auto take = [&](size_t sz) { char* r = p; p += al256(sz); return r; };
  L.Stab = (double*)take(sizeof(double) * (2 * (size_t)N + 3));
  L.lam = (double*)take(sizeof(double) * ((size_t)N + 2));
  for (int b = 0; b < 2; ++b) L.nt[b] = (double*)take(sizeof(double) * 4 * ((size_t)N + 2));
  for (int b = 0; b < 2; ++b) L.off[b] = (int*)take(sizeof(int) * (2 * ((size_t)N + 2) + 1));
  for (int b = 0; b < 2; ++b) {
    L.zY[b] = (double*)take(sizeof(double) * cap);
    L.zF[b] = (double*)take(sizeof(double) * cap);
    L.zS[b] = (double*)take(sizeof(double) * cap);
  }
  L.wY = (double*)take(sizeof(double) * cap);
  L.wF = (double*)take(sizeof(double) * cap);
  L.wS = (double*)take(sizeof(double) * cap);
  L.wGK = (long long*)take(sizeof(long long) * cap);
  L.wHK = (long long*)take(sizeof(long long) * cap);
  L.wCA = (long long*)take(sizeof(long long) * cap);
  L.wCB = (long long*)take(sizeof(long long) * cap);
  L.wN = (int*)take(sizeof(int) * cap);
  L.capZ = (int)cap;
  L.capW = (int)cap;
  return p;
}

// Carve an arena of `bytes` for an option with N steps.  Returns false when the
// arena cannot hold the node arrays and at least min_cap points per array.
OB_HD bool carve(char* base, size_t bytes, int N, int min_cap, Lay& L) {
  size_t nb = node_bytes(N) + 16 * 256;
  if (bytes < nb) return false;
  size_t cap = (bytes - nb) / ELEM_BYTES;
  if (cap > 0x3fffffff) cap = 0x3fffffff;
  if ((long long)cap < (long long)min_cap) return false;
  char* p = carve_cap(base, N, cap, L);
  return (size_t)(p - base) <= bytes;
}

// The arrays of one level's successor maximum w (and of g, h and their running
// minima): the option's global scratch, or a chunk of nodes in shared memory.
struct WBuf {
  double *Y, *F, *S;
  int* N;                 // node of each point
  long long *GK, *HK;     // keys of g = w + S^a y and h = w + S^b y
  long long *CA, *CB;     // running minima of the g keys (from the right) and h keys (from the left)
  int cap;
};

OB_HD WBuf global_wbuf(const Lay& L) {
  return WBuf{L.wY, L.wF, L.wS, L.wN, L.wGK, L.wHK, L.wCA, L.wCB, L.capW};
}

// Bytes of shared memory per point of a WBuf, and the WBuf of cap points carved at p
// (8-byte arrays first, so every array stays 8-byte aligned).
constexpr int WBUF_POINT_BYTES = 3 * 8 + 4 * 8 + 4;
OB_HD WBuf carve_wbuf(char* p, int cap) {
  WBuf w;
  w.Y = (double*)p; p += 8 * (size_t)cap;
  w.F = (double*)p; p += 8 * (size_t)cap;
  w.S = (double*)p; p += 8 * (size_t)cap;
  w.GK = (long long*)p; p += 8 * (size_t)cap;
  w.HK = (long long*)p; p += 8 * (size_t)cap;
  w.CA = (long long*)p; p += 8 * (size_t)cap;
  w.CB = (long long*)p; p += 8 * (size_t)cap;
  w.N = (int*)p;
  w.cap = cap;
  return w;
}

OB_HD double ob_inf() { return bitsd(0x7FF0000000000000LL); }

struct Em {
  double y, f, s;
};

// Value at x of the successor function piece anchored at its breakpoint k
// (k = -1: the left tail, anchored at the first breakpoint).
OB_HD double seg_eval(const double* Y, const double* F, const double* S, int k, double tailL,
                      double x) {
  return (k >= 0) ? F[k] + S[k] * (x - Y[k]) : F[0] + tailL * (x - Y[0]);
}

// ------------------------------------------------------------------ pass 1
// One union point of w = max(A, B) (A = up successor, B = down successor).
// The owner of every segment between two neighbouring union points is decided
// once, by the point at its left end (own), and handed to the point at its right
// end, which needs it as the owner just left of itself; so the two ends never
// disagree about a crossing that rounds onto a breakpoint.
struct P1 {
  double y, a, b, aL, aR, bL, bR;
  double xr, vr, sr;  // crossing before the next union point
  double xl, vl, sl;  // crossing in the left tail (first union point of a node)
  int wr;             // owner just right of y
  int own;            // owner just left of the next union point
  int wl_first;       // owner just left of y, first union point only
  int farL;           // owner of the far left (first union point only)
  bool dup, rc, lc;
  // provenance, for the adjoint: breakpoint indices used, the successors whose lines
  // meet at the crossings
  int ia, ka, ib, kb, lc_w, rc_w;
  bool fromA, aBp, bBp;
};

// q is the index in the merged breakpoint order (ties: A first).
OB_HD void p1_analyze(const double* Ay, const double* Af, const double* As, int ma, double aTL,
                      const double* By, const double* Bf, const double* Bs, int mb, double bTL,
                      int q, P1& e) {
  e.dup = e.rc = e.lc = false;
  e.own = e.wr = e.wl_first = 0;
  int lo = q - mb > 0 ? q - mb : 0, hi = q < ma ? q : ma;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (kle(Ay[mid], By[q - 1 - mid])) lo = mid + 1; else hi = mid;
  }
  const int iu = lo, id = q - lo;
  const bool fromA = iu < ma && (id >= mb || kle(Ay[iu], By[id]));
  double y;
  bool aBp, bBp;
  int ia = -1, ib = -1;
  if (fromA) {
    ia = iu;
    y = Ay[ia];
    aBp = true;
    bBp = id < mb && keq(By[id], y);
    if (bBp) ib = id;
  } else {
    ib = id;
    y = By[ib];
    bBp = true;
    if (iu > 0 && keq(Ay[iu - 1], y)) {  // already represented by A's point
      e.dup = true;
      return;
    }
    aBp = false;
  }
  const int ka = aBp ? ia : iu - 1;  // last breakpoint of A at or before y
  const int kb = bBp ? ib : id - 1;
  e.ia = ia; e.ka = ka; e.ib = ib; e.kb = kb; e.fromA = fromA; e.aBp = aBp; e.bBp = bBp;
  double a, aL, aR, b, bL, bR;
  if (aBp) {
    a = Af[ia];
    aL = ia > 0 ? As[ia - 1] : aTL;
    aR = As[ia];
  } else {
    a = seg_eval(Ay, Af, As, ka, aTL, y);
    aL = aR = (ka >= 0 ? As[ka] : aTL);
  }
  if (bBp) {
    b = Bf[ib];
    bL = ib > 0 ? Bs[ib - 1] : bTL;
    bR = Bs[ib];
  } else {
    b = seg_eval(By, Bf, Bs, kb, bTL, y);
    bL = bR = (kb >= 0 ? Bs[kb] : bTL);
  }
  e.y = y; e.a = a; e.b = b; e.aL = aL; e.aR = aR; e.bL = bL; e.bR = bR;
  // next union point
  const int na = aBp ? ia + 1 : iu;
  const int nb = bBp ? ib + 1 : id;
  const bool hasA = na < ma, hasB = nb < mb;
  bool nA = false, nB = false;
  double yn = 0.0;
  if (hasA && hasB) {
    const long long ka2 = okey(Ay[na]), kb2 = okey(By[nb]);
    if (ka2 <= kb2) { yn = Ay[na]; nA = true; }
    if (kb2 <= ka2) { yn = By[nb]; nB = true; }
  } else if (hasA) {
    yn = Ay[na];
    nA = true;
  } else if (hasB) {
    yn = By[nb];
    nB = true;
  }
  const bool hasNext = nA || nB;
  const long long kA = okey(a), kB = okey(b);
  int wr = (kA != kB) ? (kA > kB ? 0 : 1) : (klt(bR, aR) ? 0 : (klt(aR, bR) ? 1 : 0));
  if (q == 0) {  // the far left belongs to the successor with the smaller left slope
    int wl = (kA != kB) ? (kA > kB ? 0 : 1) : (klt(aL, bL) ? 0 : (klt(bL, aL) ? 1 : 0));
    const int farL = klt(aL, bL) ? 0 : (klt(bL, aL) ? 1 : wl);
    e.farL = farL;
    if (farL != wl) {
      const double vW = wl ? b : a, vO = wl ? a : b, sW = wl ? bL : aL, sO = wl ? aL : bL;
      const double x = y + (vW - vO) / (sO - sW);
      if (klt(x, y)) {
        e.lc = true;
        e.lc_w = wl;
        e.xl = x;
        e.vl = vW + sW * (x - y);
        e.sl = sW;
      } else {
        wl = farL;
      }
    }
    e.wl_first = wl;
  }
  // Does the loser overtake before the next union point?  Cheap test: who is larger
  // there; only then the crossing itself is computed.
  int wn;
  if (hasNext) {
    const double an = nA ? Af[na] : seg_eval(Ay, Af, As, ka, aTL, yn);
    const double bn = nB ? Bf[nb] : seg_eval(By, Bf, Bs, kb, bTL, yn);
    const long long kAn = okey(an), kBn = okey(bn);
    wn = (kAn != kBn) ? (kAn > kBn ? 0 : 1) : wr;
  } else {  // the far right belongs to the larger right slope
    wn = klt(bR, aR) ? 0 : (klt(aR, bR) ? 1 : wr);
  }
  int own = wr;
  if (wn != wr) {
    const double vW = wr ? b : a, vO = wr ? a : b, sW = wr ? bR : aR, sO = wr ? aR : bR;
    if (klt(sW, sO)) {  // the loser climbs faster: it overtakes at x
      const double x = y + (vW - vO) / (sO - sW);
      if (!klt(y, x)) {
        wr = own = 1 - wr;  // the crossing rounds onto y
      } else if (!hasNext || klt(x, yn)) {
        e.rc = true;
        e.rc_w = wr;
        e.xr = x;
        e.vr = vW + sW * (x - y);
        e.sr = sO;
        own = 1 - wr;
      }  // else: it rounds onto the next point, the whole segment stays with wr
    }
  }
  e.wr = wr;
  e.own = own;
}

// The piece of one successor right (left = false) or left of the union point y: with a
// breakpoint i at y, the piece right of it (or of i - 1; the tail if i = 0); else the
// piece right of its breakpoint k before y (the tail if k = -1).  Codes: a point of level
// t+1, >= 0 (the piece right of it), or -1 - (node of level t+1) for a left tail.
OB_HD int p1_side_piece(bool bp, int i, int k, int off, int tail, bool left) {
  if (bp) return left ? (i > 0 ? off + i - 1 : tail) : off + i;
  return k >= 0 ? off + k : tail;
}

// For each emission of p1_emit (same order), the successor piece whose line w follows
// right of the emitted point: after a left-tail crossing the winner's piece left of y,
// after y the winner's piece right of y, after a crossing the other side's piece right of y.
OB_HD int p1_emit_src(const P1& e, int wl, int aoff, int boff, int tailA, int tailB, int* src) {
  int n = 0;
  if (e.dup) return 0;
  if (e.lc) src[n++] = e.lc_w ? p1_side_piece(e.bBp, e.ib, e.kb, boff, tailB, true)
                              : p1_side_piece(e.aBp, e.ia, e.ka, aoff, tailA, true);
  const double sLw = wl ? e.bL : e.aL, sRw = e.wr ? e.bR : e.aR;
  if (!same_bits(sLw, sRw))
    src[n++] = e.wr ? p1_side_piece(e.bBp, e.ib, e.kb, boff, tailB, false)
                    : p1_side_piece(e.aBp, e.ia, e.ka, aoff, tailA, false);
  if (e.rc) src[n++] = e.rc_w ? p1_side_piece(e.aBp, e.ia, e.ka, aoff, tailA, false)
                              : p1_side_piece(e.bBp, e.ib, e.kb, boff, tailB, false);
  return n;
}

// Emissions of an analysed union point, given the owner just left of it.
OB_HD int p1_emit(const P1& e, int wl, Em* em) {
  int n = 0;
  if (e.dup) return 0;
  if (e.lc) em[n++] = Em{e.xl, e.vl, e.sl};
  const double sLw = wl ? e.bL : e.aL, sRw = e.wr ? e.bR : e.aR;
  if (!same_bits(sLw, sRw)) em[n++] = Em{e.y, (okey(e.a) >= okey(e.b)) ? e.a : e.b, sRw};
  if (e.rc) em[n++] = Em{e.xr, e.vr, e.sr};
  return n;
}

// ------------------------------------------------------------------ scalars
// The per-piece logic below is written for a scalar type T (double in every run) and
// a decision policy D (NoDec: decisions are taken on the values as they come).
OB_HD double val(double x) { return x; }
template <class T>
OB_HD T mk(double x);
template <>
OB_HD double mk<double>(double x) { return x; }

struct NoDec {
  OB_HD int take(int c) { return c; }
};

// ------------------------------------------------------------------ pass 3 helpers
// A line of the restriction/exercise step.  Point-slope form anchored at x0
// (exact there); an F line (a piece of w) is also exact at its right end x1.
template <class T>
struct LnT {
  T x0, v0, s;
  int icpt;  // 1: intercept form, value = v0 + s*x
  int endp;  // 1: the piece of w, also exact at the piece's right end (ex, ev below)
};

template <class T>
OB_HD T ln_eval(const LnT<T>& l, const T& x, const T& ex, const T& ev) {
  if (l.icpt) return l.v0 + l.s * x;
  if (same_bits(val(x), val(l.x0))) return l.v0;
  if (l.endp && same_bits(val(x), val(ex))) return ev;
  return l.v0 + l.s * (x - l.x0);
}

constexpr int MAXSUB = 10;

// Combine the line pi with the line qi on the sub-piece [x0, x1) (x0 may be -inf, x1
// +inf): the result is max(P, Q) (take_max) or min(P, Q) there, as one or two
// sub-pieces, returned as (x0, la) and, when split, (xb, lb).  A crossing that rounds
// onto an end leaves one line: the side of a crossing follows from the slopes (left
// of it the line of smaller slope is the larger one), so a tie at one end that
// rounding tipped the wrong way cannot misplace the piece.
template <class T, class D>
OB_HD int comb1(const LnT<T>* lines, const T& ex, const T& ev, const T& x0, const T& x1, int pi,
                int qi, bool take_max, D& dec, int& la, T& xb, int& lb) {
  la = pi;
  if (pi == qi) return 1;
  const double INF = ob_inf();
  const LnT<T>& P = lines[pi];
  const LnT<T>& Q = lines[qi];
  const bool finite0 = !same_bits(val(x0), -INF), finite1 = !same_bits(val(x1), INF);
  const long long kps = okey(val(P.s)), kqs = okey(val(Q.s));
  // outcome: 0 left winner whole, 1 right line whole, 2 left line whole, 3 split
  int outcome = 0, lw = pi;
  T p0 = mk<T>(0.0), q0 = mk<T>(0.0), p1 = mk<T>(0.0), q1 = mk<T>(0.0);
  if (finite0) { p0 = ln_eval(P, x0, ex, ev); q0 = ln_eval(Q, x0, ex, ev); }
  if (finite1) { p1 = ln_eval(P, x1, ex, ev); q1 = ln_eval(Q, x1, ex, ev); }
  const int left_line = ((kps < kqs) == take_max) ? pi : qi;
  const int right_line = (left_line == pi) ? qi : pi;
  {
    int wl, wr;  // 0 = P, 1 = Q
    if (finite0) {
      const long long a = okey(val(p0)), b = okey(val(q0));
      if (a != b) wl = ((a > b) == take_max) ? 0 : 1;
      else wl = (kps == kqs) ? 0 : (((kps > kqs) == take_max) ? 0 : 1);
    } else {
      if (kps != kqs) wl = ((kps < kqs) == take_max) ? 0 : 1;
      else { const long long a = okey(val(p1)), b = okey(val(q1)); wl = (a == b) ? 0 : (((a > b) == take_max) ? 0 : 1); }
    }
    if (finite1) {
      const long long a = okey(val(p1)), b = okey(val(q1));
      if (a != b) wr = ((a > b) == take_max) ? 0 : 1;
      else wr = (kps == kqs) ? 0 : (((kps < kqs) == take_max) ? 0 : 1);
    } else {
      if (kps != kqs) wr = ((kps > kqs) == take_max) ? 0 : 1;
      else { const long long a = okey(val(p0)), b = okey(val(q0)); wr = (a == b) ? 0 : (((a > b) == take_max) ? 0 : 1); }
    }
    lw = wl ? qi : pi;
    if (wl == wr || kps == kqs) {
      outcome = 0;
    } else {
      const double xd = finite0 ? val(x0) + (val(p0) - val(q0)) / (val(Q.s) - val(P.s))
                                : val(x1) + (val(p1) - val(q1)) / (val(Q.s) - val(P.s));
      if (!klt(val(x0), xd)) outcome = 1;
      else if (!klt(xd, val(x1))) outcome = 2;
      else outcome = 3;
    }
  }
  outcome = dec.take(outcome);
  lw = dec.take(lw);
  if (outcome == 0) { la = lw; return 1; }
  if (outcome == 1) { la = right_line; return 1; }
  if (outcome == 2) { la = left_line; return 1; }
  la = left_line;
  lb = right_line;
  xb = finite0 ? x0 + (p0 - q0) / (Q.s - P.s) : x1 + (p1 - q1) / (Q.s - P.s);
  return 2;
}

template <class T>
struct EmT {
  T y, f, s;
};

// Inputs of one piece of w (point i to point i+1, or the right tail), in the
// scalar type of the run.  Keys and flags come from the double data.
template <class T>
struct PieceIn {
  T y0, f0, s0, y1, f1;  // w at points i and i+1 (i+1 unused on the right tail)
  T cA0;                 // running minimum of g from point i (left tail line intercept)
  T cA1, cB;             // cA_{i+1}, cB_i
  T Sa, Sb, vu;          // node constants; vu = xi (seller) or -xi (buyer)
  double yu;             // kink of u
  bool head, tail, seller, anchor, Arel, Brel;
};

template <class T>
struct PieceOut {
  EmT<T> tl[3];          // emissions inside the left tail (head only)
  int ntl;
  EmT<T> first;          // candidate point at y_i
  EmT<T> m[MAXSUB];      // emissions inside the piece
  int nm;
  double last_slope, tail_slope;
  // piece() hands its emissions over in output order: left tail, first, inside, each
  // with the line (0..4 of piece()) the function follows right of the point; set_tail
  // gives the line of the far left (head only).  The pricing run keeps no lines.
  OB_HD void begin() { ntl = nm = 0; }
  OB_HD void add_tl(const EmT<T>& e, int) { tl[ntl++] = e; }
  OB_HD void set_first(const EmT<T>& e, int) { first = e; }
  OB_HD void add_m(const EmT<T>& e, int) { m[nm++] = e; }
  OB_HD void set_tail(int) {}
};

// PieceOut that also keeps the line of every emission (the adjoint's rerun of pass 3).
template <class T>
struct PieceOutL : PieceOut<T> {
  unsigned char tl_line[3], first_line, m_line[MAXSUB], tail_line;
  OB_HD void add_tl(const EmT<T>& e, int l) { tl_line[this->ntl] = (unsigned char)l; this->tl[this->ntl++] = e; }
  OB_HD void set_first(const EmT<T>& e, int l) { first_line = (unsigned char)l; this->first = e; }
  OB_HD void add_m(const EmT<T>& e, int l) { m_line[this->nm] = (unsigned char)l; this->m[this->nm++] = e; }
  OB_HD void set_tail(int l) { tail_line = (unsigned char)l; }
};

// Kinds of the line a piece of z follows (the adjoint's record of pass 3), in the top
// four bits of a code whose low 28 bits give a point of w: KW the piece of w starting at
// that point; KA, KB the line of slope -S^a (-S^b) through the point where the running
// minimum of g (h) is attained; KU3, KU4 the left and right branch of u (the point is
// the piece of w, which names the node).
enum { KW = 0, KA = 1, KB = 2, KU3 = 3, KU4 = 4 };
constexpr unsigned KSHIFT = 28, KMASK = (1u << KSHIFT) - 1;

// The restriction and the exercise step on one piece (and, for the first point
// of a node, on the left tail).
template <class T, class D, class O>
OB_HD void piece(const PieceIn<T>& in, O& out, D& dec) {
  const double INF = ob_inf();
  out.begin();
  LnT<T> lines[5];  // 0 piece of w, 1 cA line, 2 cB line, 3 u left branch, 4 u right branch
  const T yu = mk<T>(in.yu);
  lines[2] = LnT<T>{mk<T>(0.0), in.cB, -in.Sb, 1, 0};
  lines[3] = LnT<T>{yu, in.vu, -in.Sa, 0, 0};
  lines[4] = LnT<T>{yu, in.vu, -in.Sb, 0, 0};
  if (in.head) {  // left tail: v is the cA_0 line; u turns at yu if yu < y0
    lines[1] = LnT<T>{mk<T>(0.0), in.cA0, -in.Sa, 1, 0};
    const bool split = dec.take(klt(in.yu, val(in.y0)) ? 1 : 0);
    int prev_l = -1;
    for (int part = 0; part < (split ? 2 : 1); ++part) {
      const T x0 = part ? yu : mk<T>(-INF);
      const T x1 = split && !part ? yu : in.y0;
      int la, lb;
      T xb;
      const int n =
          comb1(lines, in.y1, in.f1, x0, x1, 1, part ? 4 : 3, in.seller, dec, la, xb, lb);
      for (int c = 0; c < n; ++c) {
        const int l = c ? lb : la;
        const T x = c ? xb : x0;
        if (prev_l < 0) out.set_tail(l);  // the far left
        else if (dec.take(same_bits(val(lines[l].s), val(lines[prev_l].s)) ? 0 : 1))
          out.add_tl(EmT<T>{x, ln_eval(lines[l], x, in.y1, in.f1), lines[l].s}, l);
        prev_l = l;
      }
    }
    out.tail_slope = val(lines[prev_l].s);  // just left of y0
  }
  const bool fast = dec.take((!in.tail && !in.Arel && !in.Brel &&
                              !(klt(val(in.y0), in.yu) && klt(in.yu, val(in.y1)))) ? 1 : 0);
  if (fast) {
    // common case: v = w on the piece and one branch of u covers it
    const bool leftside = klt(val(in.y0), in.yu);
    const int uq = leftside ? 3 : 4;  // the branch of u over the piece
    const T sQ = leftside ? -in.Sa : -in.Sb;
    const T q0 = in.vu + sQ * (in.y0 - yu), q1 = in.vu + sQ * (in.y1 - yu);
    const long long ks0 = okey(val(in.s0)), ksQ = okey(val(sQ));
    int outcome;  // 0: w, 1: u, 2: w then u, 3: u then w
    {
      const long long kf0 = okey(val(in.f0)), kq0 = okey(val(q0)), kf1 = okey(val(in.f1)),
                      kq1 = okey(val(q1));
      int wl, wr;  // 0 = w, 1 = u; ties go to the line that wins just right (left)
      if (kf0 != kq0) wl = ((kf0 > kq0) == in.seller) ? 0 : 1;
      else wl = (ks0 == ksQ) ? 0 : (((ks0 > ksQ) == in.seller) ? 0 : 1);
      if (kf1 != kq1) wr = ((kf1 > kq1) == in.seller) ? 0 : 1;
      else wr = (ks0 == ksQ) ? 0 : (((ks0 < ksQ) == in.seller) ? 0 : 1);
      if (wl == wr || ks0 == ksQ) {
        outcome = wl;
      } else {
        const double x = val(in.y0) + (val(in.f0) - val(q0)) / (val(sQ) - val(in.s0));
        const int left_line = ((ks0 < ksQ) == in.seller) ? 0 : 1;
        if (!klt(val(in.y0), x)) outcome = 1 - left_line;
        else if (!klt(x, val(in.y1))) outcome = left_line;
        else outcome = 2 + left_line;
      }
    }
    outcome = dec.take(outcome);
    if (outcome == 0) {
      out.set_first(EmT<T>{in.y0, in.f0, in.s0}, 0);
      out.last_slope = val(in.s0);
    } else if (outcome == 1) {
      out.set_first(EmT<T>{in.y0, q0, sQ}, uq);
      out.last_slope = val(sQ);
    } else {
      const T x = in.y0 + (in.f0 - q0) / (sQ - in.s0);
      if (outcome == 2) {  // w, then u from x
        out.set_first(EmT<T>{in.y0, in.f0, in.s0}, 0);
        out.add_m(EmT<T>{x, in.vu + sQ * (x - yu), sQ}, uq);
        out.last_slope = val(sQ);
      } else {  // u, then w from x
        out.set_first(EmT<T>{in.y0, q0, sQ}, uq);
        out.add_m(EmT<T>{x, in.f0 + in.s0 * (x - in.y0), in.s0}, 0);
        out.last_slope = val(in.s0);
      }
    }
    return;
  }
  // general case: v = min(w, cB line, cA line) on the piece as up to four sub-pieces
  // (the right tail: the cB line alone), each then split at yu and combined with u
  int vl[4];
  T vx[4];
  int nv = 1;
  vx[0] = in.y0;
  T hi;
  if (in.tail) {
    vl[0] = 2;
    hi = mk<T>(INF);
  } else {
    lines[0] = LnT<T>{in.y0, in.f0, in.s0, 0, 1};
    lines[1] = LnT<T>{mk<T>(0.0), in.cA1, -in.Sa, 1, 0};
    vl[0] = 0;
    hi = in.y1;
    if (in.Brel) {
      int la, lb;
      T xb;
      nv = comb1(lines, in.y1, in.f1, in.y0, hi, 0, 2, false, dec, la, xb, lb);
      vl[0] = la;
      if (nv == 2) { vx[1] = xb; vl[1] = lb; }
    }
    if (in.Arel) {
      int ml[4];
      T mx[4];
      int nm = 0;
      for (int k = 0; k < nv; ++k) {
        int la, lb;
        T xb;
        const int n = comb1(lines, in.y1, in.f1, vx[k], k + 1 < nv ? vx[k + 1] : hi, vl[k], 1,
                            false, dec, la, xb, lb);
        mx[nm] = vx[k]; ml[nm] = la; ++nm;
        if (n == 2) { mx[nm] = xb; ml[nm] = lb; ++nm; }
      }
      for (int k = 0; k < nm; ++k) { vx[k] = mx[k]; vl[k] = ml[k]; }
      nv = nm;
    }
  }
  int prev_l = -1;
  for (int k = 0; k < nv; ++k) {
    const T a = vx[k];
    const T b = k + 1 < nv ? vx[k + 1] : hi;
    const bool split = dec.take((klt(val(a), in.yu) && klt(in.yu, val(b))) ? 1 : 0);
    for (int part = 0; part < (split ? 2 : 1); ++part) {
      const T x0 = part ? yu : a;
      const T x1 = split && !part ? yu : b;
      int la, lb;
      T xb;
      const int qi = klt(val(x0), in.yu) ? 3 : 4;
      const int n = comb1(lines, in.y1, in.f1, x0, x1, vl[k], qi, in.seller, dec, la, xb, lb);
      for (int c = 0; c < n; ++c) {
        const int l = c ? lb : la;
        const T x = c ? xb : x0;
        if (prev_l < 0) {
          out.set_first(EmT<T>{in.y0, ln_eval(lines[l], in.y0, in.y1, in.f1), lines[l].s}, l);
        } else if (dec.take(same_bits(val(lines[l].s), val(lines[prev_l].s)) ? 0 : 1)) {
          out.add_m(EmT<T>{x, ln_eval(lines[l], x, in.y1, in.f1), lines[l].s}, l);
        }
        prev_l = l;
      }
    }
  }
  out.last_slope = val(lines[prev_l].s);
}

// ------------------------------------------------------------------ the option
// CHIP: the instantiation with the fused level step (w of chunks of nodes in on-chip
// arrays, level_fused); the plain instantiation reads and writes w in the global scratch.
// LOCAL: the passes see a window of columns of each level (a trapezoid round of the
// whole-GPU form, TcTrap): level t holds the columns [cj0, min(cjend + t, t + 1)), indexed
// from cj0 in the level arrays and the node tables; otherwise every column.
// SPLIT: pass 1 takes a range of union points that may start and end inside nodes (a share
// of a split level, TcSplit), and passes 2-3 see the w points just outside their range (the
// neighbouring shares' points at index -1 and wtot when the first and last nodes continue).
template <class Team, bool CHIP = false, bool LOCAL = false, bool SPLIT = false>
struct TcRun {
  const Team& tm;
  const Opt& o;
  const Lay& L;
  int N;
  int zeta;  // -1 put, +1 call, 0 spread
  Stats st;
  // where pass 1 reads level t+1 and pass 3 writes level t (the two banks by default)
  const double *inY, *inF, *inS;
  const int* inOff;
  double *outY, *outF, *outS;
  int* outOff;
  int outCap;
  WBuf wb;    // CHIP: where passes 1-3 keep w (chip, or the global scratch for big nodes)
  WBuf chip;  // CHIP: on-chip arrays of the fused level step
  int cj0 = 0, cjend = 0;  // LOCAL: the column window (see above)
  // SPLIT: the union points [ub, ue) of pass 1, the owner code (2 own) of the union point
  // before ub, whether the first and last nodes continue in the previous and next shares,
  // and the slope of the function just left of the first piece when the first node does
  int ub = 0, ue = 0, carry0 = 0;
  bool lcont = false, rcont = false, head_m1 = false;
  double slope0 = 0.0;

  OB_HD TcRun(const Team& tm_, const Opt& o_, const Lay& L_) : tm(tm_), o(o_), L(L_), N(o_.N) {
    zeta = (o.payoff == PAY_PUT) ? -1 : (o.payoff == PAY_CALL ? 1 : 0);
    st.upts = st.wpts = st.zpts = 0;
    st.zmax_level = 0;
    for (int c = 0; c < 4; ++c) st.hedge[c] = bitsd(0x7ff8000000000000LL);
    use_banks(N);
    if (CHIP) {
      wb = global_wbuf(L);
      chip = wb;
    }
  }

  // the arrays of w the passes use
  OB_HD double* wY() const { return CHIP ? wb.Y : L.wY; }
  OB_HD double* wF() const { return CHIP ? wb.F : L.wF; }
  OB_HD double* wS() const { return CHIP ? wb.S : L.wS; }
  OB_HD int* wN() const { return CHIP ? wb.N : L.wN; }
  OB_HD long long* wGK() const { return CHIP ? wb.GK : L.wGK; }
  OB_HD long long* wHK() const { return CHIP ? wb.HK : L.wHK; }
  OB_HD long long* wCA() const { return CHIP ? wb.CA : L.wCA; }
  OB_HD long long* wCB() const { return CHIP ? wb.CB : L.wCB; }
  OB_HD int wcap() const { return CHIP ? wb.cap : L.capW; }

  // level t reads the bank of t+1 and writes the bank of t
  OB_HD void use_banks(int t) {
    const int b1 = (t + 1) & 1, bt = t & 1;
    inY = L.zY[b1]; inF = L.zF[b1]; inS = L.zS[b1]; inOff = L.off[b1];
    outY = L.zY[bt]; outF = L.zF[bt]; outS = L.zS[bt]; outOff = L.off[bt];
    outCap = L.capZ;
  }

  // columns of level t that the level arrays hold
  OB_HD int cols(int t) const {
    if constexpr (LOCAL) {
      const int e = cjend + t;
      return (e < t + 1 ? e : t + 1) - cj0;
    } else {
      return t + 1;
    }
  }

  OB_HD void node_table(int t) { node_table_range(t, 0, cols(t) - 1); }

  // per-node constants of level t for the nodes jlo <= j <= jhi
  OB_HD void node_table_range(int t, int jlo, int jhi) {
    const int lane = tm.lane();
    double* nt = L.nt[t & 1];
    const double lam = L.lam[t];
    const double kt = (t == 0) ? 0.0 : o.k;
    for (int j = jlo + lane; j <= jhi; j += Team::W) {
      const int ja = LOCAL ? j + cj0 : j;  // the column in the tree
      const double S = L.Stab[2 * ja - t + N + 1];
      const double Sl = S * lam;
      nt[4 * j] = Sl * (1.0 + kt);
      nt[4 * j + 1] = Sl * (1.0 - kt);
      double xi;
      if (o.payoff == PAY_PUT) xi = o.K;
      else if (o.payoff == PAY_CALL) xi = -o.K;
      else xi = fmax(S - o.K, 0.0) - fmax(S - o.K2, 0.0);
      nt[4 * j + 2] = xi * lam;
    }
  }

  // union start of node (p, j) of level t; j in [0, t+1]
  OB_HD int ustart(const int* o1, int W1, int UB1, int p, int j) const {
    const int* op = o1 + p * W1;
    return (p ? UB1 : 0) + (op[j] - op[0]) + (op[j + 1] - op[1]);
  }

  // union start of node n (seller nodes 0..t, then buyer nodes) of level t; n in [0, 2(t+1)]
  OB_HD int ustart_node(int t, int n) const {
    const int W1 = cols(t + 1), W0 = cols(t);
    const int UB1 = ustart(inOff, W1, 0, 0, W0);
    const int p = n >= W0 ? 1 : 0;
    return ustart(inOff, W1, UB1, p, n - p * W0);
  }

  // SPLIT: 2 * (owner just left of the next union point) of the last union point before q
  // that is not a duplicate, for q inside node n of level t (q > its first union point); the
  // carry that pass 1 would hand across from the union points before q.
  OB_HD int own_before(int t, int n, int q) const {
    const int W1 = cols(t + 1), W0 = cols(t);
    const int* o1 = inOff;
    const double* nt1 = L.nt[(t + 1) & 1];
    const int UB1 = ustart(o1, W1, 0, 0, W0);
    const int p = n >= W0 ? 1 : 0;
    const int j = n - p * W0;
    const int* op = o1 + p * W1;
    const int aoff = op[j + 1], ma = op[j + 2] - aoff, boff = op[j], mb = aoff - boff;
    int ql = q - 1 - ustart(o1, W1, UB1, p, j);
    P1 e;
    p1_analyze(inY + aoff, inF + aoff, inS + aoff, ma, -nt1[4 * (j + 1)], inY + boff, inF + boff,
               inS + boff, mb, -nt1[4 * j], ql, e);
    if (e.dup && ql > 0)  // duplicates are never adjacent, and never a node's first point
      p1_analyze(inY + aoff, inF + aoff, inS + aoff, ma, -nt1[4 * (j + 1)], inY + boff, inF + boff,
                 inS + boff, mb, -nt1[4 * j], ql - 1, e);
    return 2 * e.own;
  }

  // pass 1: w = max(z_up, z_down) for the nodes n0 <= n < n1 of level t (n1 < 0: all
  // nodes); w of node n0 starts at position 0.  Returns false on overflow.
  // PROV (the adjoint's rerun): wsrc[i] receives the successor piece whose line w follows
  // right of point i of w, wtail[node] that of w's left tail (p1_side_piece codes).
  template <bool PROV = false>
  OB_HD bool pass1(int t, int& wtot, int& utot, int n0 = 0, int n1 = -1, int* wsrc = nullptr,
                   int* wtail = nullptr) {
    const int lane = tm.lane();
    const int b1 = (t + 1) & 1;
    const int W1 = cols(t + 1), W0 = cols(t), nNodes = 2 * W0;
    const int* o1 = inOff;
    const double *Y1 = inY, *F1 = inF, *S1 = inS;
    const double* nt1 = L.nt[b1];
    const int UB1 = ustart(o1, W1, 0, 0, W0);
    if (n1 < 0) n1 = nNodes;
    const int u0 = SPLIT ? ub : ustart_node(t, n0);
    const int Utot = SPLIT ? ue : ustart_node(t, n1);  // end of the range
    utot = Utot - u0;
    int ncur = n0, wpos = 0, carry_own = SPLIT ? carry0 : 0;  // 2*own of the last non-duplicate point
    bool ovf = false;
    for (int base = u0; base < Utot; base += Team::W) {
      const int q = base + lane;
      const int nl = ncur + lane;
      int nend = 0x7fffffff;
      if (nl < n1) {
        const int p = nl >= W0 ? 1 : 0;
        nend = ustart(o1, W1, UB1, p, nl - p * W0 + 1);
      }
      // node of q: number of node ends <= q among those loaded (ends are increasing)
      int pos, nend_le;
      tm.count_le2(nend, q, base + Team::W, pos, nend_le);
      const int ncur_next = ncur + nend_le;
      Em em[3];
      P1 e;
      e.dup = true;
      e.own = 0;  // lanes past the end hand a defined code on
      int cnt = 0, node = ncur + pos, ql = -1;
      int aoff = 0, boff = 0, tailA = 0, tailB = 0;
      if (q < Utot) {
        const int p = node >= W0 ? 1 : 0;
        const int j = node - p * W0;
        ql = q - ustart(o1, W1, UB1, p, j);
        const int* op = o1 + p * W1;
        aoff = op[j + 1];
        const int ma = op[j + 2] - aoff;
        boff = op[j];
        const int mb = aoff - boff;
        tailA = -1 - (p * W1 + j + 1);
        tailB = -1 - (p * W1 + j);
        p1_analyze(Y1 + aoff, F1 + aoff, S1 + aoff, ma, -nt1[4 * (j + 1)], Y1 + boff, F1 + boff,
                   S1 + boff, mb, -nt1[4 * j], ql, e);
      }
      // owner of the segment ending at this point: that of the previous union point,
      // looking past a duplicate (duplicates are never adjacent); encoded 2*own + dup
      int m1, m2, l1, l2;
      const int code = (q < Utot && e.dup) ? 1 : 2 * e.own;
      tm.look2(code, carry_own, carry_own, m1, m2, l1, l2);
      const int v2 = (m1 & 1) ? (m2 >> 1) : (m1 >> 1);
      carry_own = (l1 & 1) ? l2 : l1;
      if (q < Utot) cnt = p1_emit(e, ql == 0 ? e.wl_first : v2, em);
      int src[3];
      if (PROV && q < Utot) {
        p1_emit_src(e, ql == 0 ? e.wl_first : v2, aoff, boff, tailA, tailB, src);
        if (ql == 0) wtail[node] = e.farL ? tailB : tailA;
      }
      int total;
      const int pre = tm.excl_sum(cnt, total);
      const int p0 = wpos + pre;
      if (p0 + cnt <= wcap()) {
        for (int c = 0; c < cnt; ++c) {
          wY()[p0 + c] = em[c].y;
          wF()[p0 + c] = em[c].f;
          wS()[p0 + c] = em[c].s;
          wN()[p0 + c] = node;
          if (PROV) wsrc[p0 + c] = src[c];
        }
      } else if (cnt > 0) {
        ovf = true;
      }
      wpos += total;
      ncur = ncur_next;
    }
    wtot = wpos;
    return !(tm.any(ovf) || wpos > wcap());
  }

  // pass 2: g, h and the per-node running minima of their keys (and, for the
  // adjoint, the index where each minimum is attained)
  template <bool TRACK = false>
  OB_HD void pass2(int t, int wtot, int* argA = nullptr, int* argB = nullptr) {
    const int lane = tm.lane();
    const int W0 = cols(t);
    const double* nt = L.nt[t & 1];
    const long long KMAX = 0x7fffffffffffffffLL;
    long long carry = KMAX;
    int carry_i = 0;
    for (int base = 0; base < wtot; base += Team::W) {
      const int i = base + lane;
      const bool ok = i < wtot;
      const int n = ok ? wN()[i] : -1;
      const bool head = ok && (i == 0 || wN()[i - 1] != n);
      long long hk = KMAX;
      if (ok) {
        const int j = n >= W0 ? n - W0 : n;
        const double y = wY()[i], f = wF()[i];
        const double g = f + nt[4 * j] * y, h = f + nt[4 * j + 1] * y;
        wGK()[i] = okey(g);
        hk = okey(h);
        wHK()[i] = hk;
      }
      if (TRACK) {
        int ix = i;
        tm.seg_argmin(hk, ix, head, carry, carry_i);
        if (ok) { wCB()[i] = hk; argB[i] = ix; }
      } else {
        const long long v = tm.seg_min(hk, head, carry);
        if (ok) wCB()[i] = v;
      }
    }
    tm.sync();
    carry = KMAX;
    carry_i = 0;
    const int ntiles = (wtot + Team::W - 1) / Team::W;
    for (int tile = ntiles - 1; tile >= 0; --tile) {
      const int i = tile * Team::W + (Team::W - 1 - lane);
      const bool ok = i < wtot;
      const int n = ok ? wN()[i] : -1;
      const bool head = ok && (i + 1 == wtot || wN()[i + 1] != n);
      long long gk = ok ? wGK()[i] : KMAX;
      if (TRACK) {
        int ix = i;
        tm.seg_argmin(gk, ix, head, carry, carry_i);
        if (ok) { wCA()[i] = gk; argA[i] = ix; }
      } else {
        const long long v = tm.seg_min(gk, head, carry);
        if (ok) wCA()[i] = v;
      }
    }
    tm.sync();
  }

  // inputs of the piece starting at point i of w (level t)
  OB_HD void load_piece(int t, int i, int wtot, PieceIn<double>& in, int& node) const {
    const int W0 = cols(t);
    const double* nt = L.nt[t & 1];
    node = wN()[i];
    if constexpr (SPLIT) {
      if (i < 0) {  // the previous share's last point: its head flag came with it
        in.head = head_m1;
        in.tail = false;
      } else {
        in.head = (i == 0) ? !lcont : wN()[i - 1] != node;
        in.tail = (i + 1 == wtot) ? !rcont : wN()[i + 1] != node;
      }
    } else {
      in.head = (i == 0 || wN()[i - 1] != node);
      in.tail = (i + 1 == wtot || wN()[i + 1] != node);
    }
    const int p = node >= W0 ? 1 : 0;
    const int j = node - p * W0;
    in.Sa = nt[4 * j];
    in.Sb = nt[4 * j + 1];
    const double xi = nt[4 * j + 2];
    in.seller = (p == 0);
    in.yu = in.seller ? (double)zeta : -(double)zeta;
    in.vu = in.seller ? xi : -xi;
    in.anchor = in.head && same_bits(in.Sa, in.Sb);
    in.y0 = wY()[i];
    in.f0 = wF()[i];
    in.s0 = wS()[i];
    const long long cB = wCB()[i];
    in.cB = unkey(cB);
    in.cA0 = unkey(wCA()[i]);
    in.Arel = in.Brel = false;
    in.y1 = in.f1 = in.cA1 = 0.0;
    if (!in.tail) {
      in.y1 = wY()[i + 1];
      in.f1 = wF()[i + 1];
      const long long cA1 = wCA()[i + 1];
      in.cA1 = unkey(cA1);
      const long long g0 = wGK()[i], g1 = wGK()[i + 1];
      const long long h0 = wHK()[i], h1 = wHK()[i + 1];
      // the cA line lies above w on the whole piece iff g <= cA_{i+1} at both ends;
      // the cB line iff h <= cB_i at both ends (then that side of v equals w)
      in.Arel = !(g1 == cA1 && g0 <= cA1);
      in.Brel = !(h0 == cB && h1 <= cB);
    }
  }

  // SPLIT: the slope of z just left of w point 0 when its node continues from the previous
  // share: the last slope of the piece that starts at that share's last point (index -1)
  OB_HD double slope_before(int t) const {
    PieceIn<double> in;
    int node;
    load_piece(t, -1, 0, in, node);
    PieceOut<double> po;
    po.ntl = po.nm = 0;
    po.first = EmT<double>{0.0, 0.0, 0.0};
    po.last_slope = po.tail_slope = 0.0;
    NoDec nd;
    piece(in, po, nd);
    return po.last_slope;
  }

  // pass 3: restriction and exercise for every piece of w; writes level t, the
  // points from position zbase on (w of a chunk of nodes: its first node's points)
  // PROV (the adjoint's rerun): zsrc[p] receives the line (KW..KU4 code) the function
  // follows right of emitted point p, ztail[node] that of its left tail; argA, argB are the
  // points where pass 2's running minima are attained.
  template <bool PROV = false>
  OB_HD bool pass3(int t, int wtot, int& ztot, int zbase = 0, unsigned* zsrc = nullptr,
                   unsigned* ztail = nullptr, const int* argA = nullptr, const int* argB = nullptr) {
    const int lane = tm.lane();
    const int nNodes = 2 * cols(t);
    int* off = outOff;
    double* Yz = outY;
    double* Fz = outF;
    double* Sz = outS;
    int zpos = zbase;
    bool ovf = false;
    double carry_slope = SPLIT ? slope0 : 0.0;
    for (int base = 0; base < wtot; base += Team::W) {
      const int i = base + lane;
      const bool ok = i < wtot;
      typename std::conditional<PROV, PieceOutL<double>, PieceOut<double>>::type po;
      po.ntl = po.nm = 0;
      po.first = EmT<double>{0.0, 0.0, 0.0};
      po.last_slope = po.tail_slope = 0.0;
      bool head = false, anchor = false;
      int node = -1;
      if (ok) {
        PieceIn<double> in;
        load_piece(t, i, wtot, in, node);
        head = in.head;
        anchor = in.anchor;
        NoDec nd;
        piece(in, po, nd);
      }
      const double last_slope = po.last_slope;
      // slope of z just left of this piece's first point
      double tile_last_slope;
      double prev = tm.prev_last(last_slope, carry_slope, tile_last_slope);
      if (head) prev = po.tail_slope;
      const int emit_first = (ok && (anchor || !same_bits(prev, po.first.s))) ? 1 : 0;
      const int nout = ok ? po.ntl + emit_first + po.nm : 0;
      int total;
      const int pre = tm.excl_sum(nout, total);
      const int p0 = zpos + pre;
      if (ok && head) off[node] = p0;
      if (ok) {
        if (p0 + nout <= outCap) {
          int w = p0;
          for (int c = 0; c < po.ntl; ++c, ++w) { Yz[w] = po.tl[c].y; Fz[w] = po.tl[c].f; Sz[w] = po.tl[c].s; }
          if (emit_first) { Yz[w] = po.first.y; Fz[w] = po.first.f; Sz[w] = po.first.s; ++w; }
          for (int c = 0; c < po.nm; ++c, ++w) { Yz[w] = po.m[c].y; Fz[w] = po.m[c].f; Sz[w] = po.m[c].s; }
          if constexpr (PROV) {
            // lines 0..4 of piece(): the piece of w, the cA line (cA_i in the left tail,
            // cA_{i+1} inside the piece), the cB line, the two branches of u
            auto code = [&](int l, bool left_tail) -> unsigned {
              if (l == 0) return ((unsigned)KW << KSHIFT) | (unsigned)i;
              if (l == 1) return ((unsigned)KA << KSHIFT) | (unsigned)(left_tail ? argA[i] : argA[i + 1]);
              if (l == 2) return ((unsigned)KB << KSHIFT) | (unsigned)argB[i];
              return ((unsigned)(l == 3 ? KU3 : KU4) << KSHIFT) | (unsigned)i;
            };
            int v = p0;
            for (int c = 0; c < po.ntl; ++c, ++v) zsrc[v] = code(po.tl_line[c], true);
            if (emit_first) zsrc[v++] = code(po.first_line, false);
            for (int c = 0; c < po.nm; ++c, ++v) zsrc[v] = code(po.m_line[c], false);
            if (head) ztail[node] = code(po.tail_line, true);
          }
        } else if (nout > 0) {
          ovf = true;
        }
      }
      carry_slope = tile_last_slope;
      zpos += total;
    }
    if (lane == 0) off[nNodes] = zpos;
    ztot = zpos - zbase;
    return !(tm.any(ovf) || zpos > outCap);
  }

  // first node n of level t (0 <= n <= 2(t+1)) whose union start is >= target: each
  // round the team probes W evenly spaced nodes of the bracket at once and keeps the
  // gap that holds it
  OB_HD int node_at(int t, long long target) const {
    int lo = 0, hi = 2 * cols(t);  // the answer lies in [lo, hi]
    while (lo < hi) {
      const int step = (hi - lo + Team::W - 1) / Team::W;
      const int n = lo + tm.lane() * step;
      const bool below = n < hi && (long long)ustart_node(t, n) < target;
      const int cnt = tm.count(below);  // the probes below the answer come first
      if (cnt == 0) break;              // lo itself is at or above it
      const int nhi = lo + cnt * step;
      lo = lo + (cnt - 1) * step + 1;
      if (nhi < hi) hi = nhi;
    }
    return lo;
  }

  // One level with w on chip: the level's nodes in chunks of whole nodes whose merged
  // successor points number at most chip.cap; passes 1-3 run per chunk with w, the keys
  // of g and h and their running minima in `chip` (shared memory), and only z is written
  // to the level's bank.  A node too large for the chip arrays, or a chunk whose w
  // outgrows them (crossings add points), runs on the global arrays instead.  The
  // running minima restart at every node, so chunks of whole nodes give the same
  // numbers as the one-pass level.  Returns false on overflow of the global arrays.
  OB_HD bool level_fused(int t, int& utot, int& wtot, int& ztot) {
    static_assert(CHIP, "the fused level step needs the on-chip instantiation");
    const int nNodes = 2 * cols(t);
    const WBuf gw = global_wbuf(L);
    const int cap = chip.cap - chip.cap / 8;  // merged points per chunk: room for crossings
    int zpos = 0, n0 = 0;
    utot = wtot = 0;
    while (n0 < nNodes) {
      const long long u0 = ustart_node(t, n0);
      int n1 = (u0 + cap >= (long long)ustart_node(t, nNodes)) ? nNodes : node_at(t, u0 + cap + 1) - 1;
      bool on_chip = true;
      if (n1 <= n0) {  // node n0 alone has more than cap merged points
        n1 = n0 + 1;
        on_chip = false;
      }
      int wt = 0, ut = 0, zt = 0;
      if (on_chip) {
        wb = chip;
        if (!pass1(t, wt, ut, n0, n1)) on_chip = false;
      }
      if (!on_chip) {
        wb = gw;
        if (!pass1(t, wt, ut, n0, n1)) { wb = gw; return false; }
      }
      pass2(t, wt);
      const bool ok = pass3(t, wt, zt, zpos);
      wb = gw;
      if (!ok) return false;
      utot += ut;
      wtot += wt;
      zpos += zt;
      n0 = n1;
    }
    ztot = zpos;
    return true;
  }

  // value at y = 0 of node n of level 0 (bank 0)
  OB_HD double root_value(int n) const {
    const int b = L.off[0][n], e = L.off[0][n + 1];
    const double tailL = -L.nt[0][0];
    if (e <= b) return 0.0;
    if (!klt(L.zY[0][b], 0.0)) return L.zF[0][b] + tailL * (0.0 - L.zY[0][b]);
    int k = b;
    while (k + 1 < e && kle(L.zY[0][k + 1], 0.0)) ++k;
    return L.zF[0][k] + L.zS[0][k] * (0.0 - L.zY[0][k]);
  }

  // The hedge at the root (Section 3: rebalancing at t = 0, where S^a = S^b = S0).  For the
  // seller's node (0) and the buyer's (1) of level 0, the point of w_0 where
  // g = w_0 + S0 lambda_0 y is least (the rightmost among equal keys): the stock holding a
  // hedger with no stock moves to, attaining v_0(0) = min g; and whether immediate
  // exercise sets the ask (u_0(0) > v_0(0)) or is the buyer's choice (u_0(0) < v_0(0)).
  // Needs w_0, its g keys and wtot of level 0 in the arrays the passes used.
  OB_HD void root_hedge(int wtot) {
    const double* nt = L.nt[0];
    const double uS = nt[2] + (double)zeta * nt[0];  // seller's u_0(0) lambda_0: xi + zeta S0
    for (int p = 0; p < 2; ++p) {
      long long cv = KMAXLL;
      int ci = -1;
      for (int base = 0; base < wtot; base += Team::W) {
        const int i = base + tm.lane();
        const bool ok = i < wtot && wN()[i] == p;
        long long gk = ok ? wGK()[i] : KMAXLL;
        int ix = ok ? i : -1;
        tm.seg_argmin(gk, ix, false, cv, ci);
      }
      const long long ku = okey(p == 0 ? uS : -uS);
      st.hedge[p] = ci >= 0 ? wY()[ci] : bitsd(0x7ff8000000000000LL);
      st.hedge[2 + p] = (p == 0 ? ku > cv : ku < cv) ? 1.0 : 0.0;
    }
  }

  // Full induction for one option; returns a status code, writes ask and bid.
  OB_HD int run(double& ask, double& bid) {
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
    // level N+1: payoff (0,0) for both parties: one point (0, 0, -S^b)
    {
      const int b = (N + 1) & 1, W = N + 2;
      node_table(N + 1);
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
    int wtot = 0;
    for (int t = N; t >= 0; --t) {
      use_banks(t);
      node_table(t);
      tm.sync();
      int ztot = 0, utot = 0;
      wtot = 0;
      if constexpr (CHIP) {
        if (!level_fused(t, utot, wtot, ztot)) return ST_CAPACITY;
      } else {
        if (!pass1(t, wtot, utot)) return ST_CAPACITY;
        pass2(t, wtot);
        if (!pass3(t, wtot, ztot)) return ST_CAPACITY;
      }
      st.upts += utot;
      st.wpts += wtot;
      st.zpts += ztot;
      if (ztot > st.zmax_level) st.zmax_level = ztot;
    }
    if constexpr (!CHIP) root_hedge(wtot);  // the fused step keeps w_0 in its chunk arrays
    const double lam0 = L.lam[0];
    ask = root_value(0) / lam0;
    bid = -root_value(1) / lam0;
    return ST_OK;
  }
};

// ------------------------------------------------------------------ one option, G teams
// The level step split over G teams (CTAs) that share the level functions.  Team c
// of G takes the nodes whose merged successor points fall in the c-th G-quantile of
// the level's union (whole nodes), runs the three passes into its private arrays,
// and, once every team's count is known, copies its points to their place in the
// shared level and rewrites the node offsets.  The caller puts a barrier of all G
// teams between compute() and publish() and after publish().  Every node is
// computed by the same element-wise code as in the one-team run, so the results
// are the same bit for bit.
struct GroupLay {
  double *zY[2], *zF[2], *zS[2];
  int* off[2];
  int capZ;
};

// Bytes of the shared level arrays for N steps and cap points per bank.
OB_HD size_t group_shared_bytes(int N, size_t cap) {
  return 2 * al256(sizeof(int) * (2 * ((size_t)N + 2) + 1)) + 6 * al256(sizeof(double) * cap);
}

// Carve the shared level arrays from `bytes` at base; false if fewer than min_cap points fit.
OB_HD bool carve_group_shared(char* base, size_t bytes, int N, int min_cap, GroupLay& S) {
  const size_t fixed = 2 * al256(sizeof(int) * (2 * ((size_t)N + 2) + 1)) + 6 * 256;
  if (bytes < fixed) return false;
  size_t cap = (bytes - fixed) / (6 * sizeof(double));
  if (cap > 0x3fffffff) cap = 0x3fffffff;
  if ((long long)cap < (long long)min_cap) return false;
  char* p = base;
  auto take = [&](size_t sz) { char* r = p; p += al256(sz); return r; };
  for (int b = 0; b < 2; ++b) S.off[b] = (int*)take(sizeof(int) * (2 * ((size_t)N + 2) + 1));
  for (int b = 0; b < 2; ++b) {
    S.zY[b] = (double*)take(sizeof(double) * cap);
    S.zF[b] = (double*)take(sizeof(double) * cap);
    S.zS[b] = (double*)take(sizeof(double) * cap);
  }
  S.capZ = (int)cap;
  return (size_t)(p - base) <= bytes;
}

template <class Team>
struct TcGroup {
  Lay L;           // private arrays; the level banks and offsets point at the shared ones
  TcRun<Team> R;
  int G, c;
  double *zpY, *zpF, *zpS;  // private output of the level (one of the carved banks)
  int* poff;                // private node offsets of the level
  int capP;
  int n0, n1, ztot;         // this team's nodes and point count of the current level

  OB_HD static Lay merge(const Lay& Lp, const GroupLay& S) {
    Lay L = Lp;
    for (int b = 0; b < 2; ++b) {
      L.zY[b] = S.zY[b]; L.zF[b] = S.zF[b]; L.zS[b] = S.zS[b]; L.off[b] = S.off[b];
    }
    L.capZ = S.capZ;
    return L;
  }

  OB_HD TcGroup(const Team& tm, const Opt& o, const Lay& Lp, const GroupLay& S, int G_, int c_)
      : L(merge(Lp, S)), R(tm, o, L), G(G_), c(c_), zpY(Lp.zY[0]), zpF(Lp.zF[0]), zpS(Lp.zS[0]),
        poff(Lp.off[0]), capP(Lp.capZ), n0(0), n1(0), ztot(0) {}

  // tree constants, the leaf level (written by team 0); a status every team agrees on
  OB_HD int begin() {
    const Team& tm = R.tm;
    const Opt& o = R.o;
    const int N = R.N, lane = tm.lane();
    const double dt = o.T / N;
    const double u = exp(o.sigma * sqrt(dt));
    const double r = exp(o.R * dt);
    const double d = 1.0 / u;
    if (!(d < r && r < u)) return ST_ARBITRAGE;
    if (2 * (N + 2) > L.capZ) return ST_CAPACITY;
    for (int e = lane; e < 2 * N + 3; e += Team::W) L.Stab[e] = o.S0 * pow(u, (double)(e - (N + 1)));
    for (int t = lane; t <= N + 1; t += Team::W) L.lam[t] = pow(r, (double)(N + 1 - t));
    tm.sync();
    const int b = (N + 1) & 1, W = N + 2;
    R.node_table(N + 1);
    tm.sync();
    if (c == 0) {
      for (int n = lane; n < 2 * W; n += Team::W) {
        const int j = n >= W ? n - W : n;
        L.off[b][n] = n;
        L.zY[b][n] = 0.0;
        L.zF[b][n] = 0.0;
        L.zS[b][n] = -L.nt[b][4 * j + 1];
      }
      if (lane == 0) L.off[b][2 * W] = 2 * W;
    }
    tm.sync();
    return ST_OK;
  }

  // this team's share of level t, into the private arrays; false on overflow
  OB_HD bool compute(int t) {
    const Team& tm = R.tm;
    R.use_banks(t);
    const int nNodes = 2 * (t + 1), W0 = t + 1;
    const long long Utot = R.ustart_node(t, nNodes);
    n0 = (c == 0) ? 0 : R.node_at(t, (Utot * c + G - 1) / G);
    n1 = (c == G - 1) ? nNodes : R.node_at(t, (Utot * (c + 1) + G - 1) / G);
    // node constants of this share only: level t for its nodes j, level t+1 for j, j+1
    // (a share that straddles the seller/buyer boundary needs two intervals of j)
    if (n0 < n1) {
      const int s_lo = n0, s_hi = (n1 < W0 ? n1 : W0) - 1;               // seller nodes
      const int b_lo = (n0 > W0 ? n0 : W0) - W0, b_hi = n1 - 1 - W0;      // buyer nodes
      if (s_lo <= s_hi) {
        R.node_table_range(t, s_lo, s_hi);
        R.node_table_range(t + 1, s_lo, s_hi + 1);
      }
      if (b_lo <= b_hi) {
        R.node_table_range(t, b_lo, b_hi);
        R.node_table_range(t + 1, b_lo, b_hi + 1);
      }
    }
    tm.sync();
    R.outY = zpY; R.outF = zpF; R.outS = zpS; R.outOff = poff; R.outCap = capP;
    int wtot = 0, utot = 0;
    ztot = 0;
    if (!R.pass1(t, wtot, utot, n0, n1)) return false;
    R.st.upts += utot;
    R.pass2(t, wtot);
    if (!R.pass3(t, wtot, ztot)) return false;
    R.st.wpts += wtot;
    R.st.zpts += ztot;
    return true;
  }

  // place this team's points of level t in the shared bank; cnt[g] = points of team g.
  // False when the level outgrows the shared bank (every team sees the same).
  OB_HD bool publish(int t, const int* cnt) {
    const Team& tm = R.tm;
    const int lane = tm.lane();
    long long pre = 0, total = 0;
    for (int g = 0; g < G; ++g) {
      if (g < c) pre += cnt[g];
      total += cnt[g];
    }
    if (total > L.capZ) return false;
    const int bt = t & 1;
    double *Y = L.zY[bt], *F = L.zF[bt], *S = L.zS[bt];
    int* off = L.off[bt];
    const int p = (int)pre;
    for (int i = lane; i < ztot; i += Team::W) {
      Y[p + i] = zpY[i];
      F[p + i] = zpF[i];
      S[p + i] = zpS[i];
    }
    for (int n = n0 + lane; n < n1; n += Team::W) off[n] = p + poff[n];
    if (c == 0 && lane == 0) off[2 * (t + 1)] = (int)total;
    if ((int)total > R.st.zmax_level) R.st.zmax_level = (int)total;
    tm.sync();
    return true;
  }

  // ask and bid from the shared level 0 (after the last publish and barrier); the node table
  // of level 0 is this team's own (a share of split nodes may not have held node 0)
  OB_HD void root(double& ask, double& bid) {
    R.node_table_range(0, 0, 0);
    R.tm.sync();
    const double lam0 = L.lam[0];
    ask = R.root_value(0) / lam0;
    bid = -R.root_value(1) / lam0;
  }
};

// ------------------------------------------------------------------ one option, trapezoid rounds
// A round of the whole-GPU form for levels light enough that a level step is latency, not
// work: from the complete shared level B, team c of Ga takes the columns [j0, j1) of level
// B - D, copies the window [j0, min(j1 + D, B + 1)) of level B (both parties) into its
// private arrays and computes the D levels below it there, each one column narrower on the
// right (node (t, j) needs (t+1, j) and (t+1, j+1)); the columns right of j1 are computed by
// the next team as well (the halo).  So the teams meet twice per round (counts, copy)
// instead of twice per level.  The results are the same bits as a level at a time: every
// node comes out of the same element-wise code from the same successors.
template <class Team>
struct TcTrap {
  Lay Lp;                    // private arrays (both banks)
  TcRun<Team, false, true> R;
  GroupLay S;
  int nS = 0, nB = 0;        // points of the round's output level: seller and buyer columns
  int j0 = 0, j1 = 0;        // output columns of the round (none when j0 >= j1)

  OB_HD TcTrap(const Team& tm, const Opt& o, const Lay& Lp_, const GroupLay& S_)
      : Lp(Lp_), R(tm, o, Lp), S(S_) {}

  // points of the complete level B in its columns below j (seller and buyer)
  OB_HD long long col_points(int B, int j) const {
    const int* so = S.off[B & 1];
    const int W = B + 1;
    return (long long)so[j] + so[W + j] - so[W];
  }

  // first column j in [0, cols] of level B with col_points(B, j) >= target: each round the
  // team probes W evenly spaced columns of the bracket and keeps the gap that holds it
  OB_HD int col_at(int B, int cols, long long target) const {
    const Team& tm = R.tm;
    int lo = 0, hi = cols;
    while (lo < hi) {
      const int step = (hi - lo + Team::W - 1) / Team::W;
      const int j = lo + tm.lane() * step;
      const bool below = j < hi && col_points(B, j) < target;
      const int cnt = tm.count(below);
      if (cnt == 0) break;
      const int nhi = lo + cnt * step;
      lo = lo + (cnt - 1) * step + 1;
      if (nhi < hi) hi = nhi;
    }
    return lo;
  }

  // A round from the complete level B (B >= 1): D levels (B-1 .. B-D, at most Dmax), Ga
  // active teams of G (at least 2D output columns each on average), and team c's output
  // columns [a, b): the c-th Ga-quantile of level B's points over the output columns (every
  // team computes the same bounds).
  OB_HD void plan(int B, int Dmax, int G, int c, int& D, int& Ga, int& a, int& b) const {
    D = B < Dmax ? B : Dmax;
    const int cout = B - D + 1;
    Ga = cout / (2 * D);
    if (Ga < 1) Ga = 1;
    if (Ga > G) Ga = G;
    const long long tot = col_points(B, cout);
    a = (c == 0) ? 0 : (c < Ga ? col_at(B, cout, tot * c / Ga) : cout);
    b = (c >= Ga - 1) ? cout : col_at(B, cout, tot * (c + 1) / Ga);
  }

  // this team's window of levels B-1 .. B-D into its private banks; false on overflow
  OB_HD bool compute(int B, int D, int a, int b) {
    const Team& tm = R.tm;
    const int lane = tm.lane();
    j0 = a;
    j1 = b;
    nS = nB = 0;
    if (j0 >= j1) return true;  // idle this round
    R.cj0 = j0;
    R.cjend = j1 + D - B;
    // the window of level B, seller columns then buyer columns, offsets from 0
    const int W = B + 1, cl = R.cols(B), je = j0 + cl, pb = B & 1;
    const int* so = S.off[pb];
    const int bs = so[j0], ns = so[je] - bs, bb = so[W + j0], nb = so[W + je] - bb;
    if (ns + nb > Lp.capZ) return false;
    double *Y = Lp.zY[pb], *F = Lp.zF[pb], *Sl = Lp.zS[pb];
    const double *SY = S.zY[pb], *SF = S.zF[pb], *SS = S.zS[pb];
    int* po = Lp.off[pb];
    for (int i = lane; i < ns; i += Team::W) {
      Y[i] = SY[bs + i];
      F[i] = SF[bs + i];
      Sl[i] = SS[bs + i];
    }
    for (int i = lane; i < nb; i += Team::W) {
      Y[ns + i] = SY[bb + i];
      F[ns + i] = SF[bb + i];
      Sl[ns + i] = SS[bb + i];
    }
    for (int k = lane; k < cl; k += Team::W) po[k] = so[j0 + k] - bs;
    for (int k = lane; k <= cl; k += Team::W) po[cl + k] = ns + so[W + j0 + k] - bb;
    R.node_table(B);  // the successors' tails of the first level
    tm.sync();
    for (int t = B - 1; t >= B - D; --t) {
      R.use_banks(t);
      R.node_table(t);
      tm.sync();
      int wtot = 0, utot = 0, ztot = 0;
      if (!R.pass1(t, wtot, utot)) return false;
      R.pass2(t, wtot);
      if (!R.pass3(t, wtot, ztot)) return false;
      R.st.upts += utot;
      R.st.wpts += wtot;
      R.st.zpts += ztot;
    }
    const int bt = (B - D) & 1, cw = j1 - j0;
    nS = Lp.off[bt][cw];
    nB = Lp.off[bt][2 * cw] - nS;
    return true;
  }

  // place this team's output columns of level T in the shared bank; cs[g], cb[g]: the
  // seller and buyer points of team g of G (0 for idle teams).  False when the level
  // outgrows the shared bank (every team sees the same).
  OB_HD bool publish(int T, int G, int c, const int* cs, const int* cb) {
    const Team& tm = R.tm;
    const int lane = tm.lane();
    long long preS = 0, preB = 0, totS = 0, totB = 0;
    for (int g = 0; g < G; ++g) {
      if (g < c) {
        preS += cs[g];
        preB += cb[g];
      }
      totS += cs[g];
      totB += cb[g];
    }
    if (totS + totB > S.capZ) return false;
    const int bt = T & 1, W = T + 1, cw = j1 - j0;
    double *Y = S.zY[bt], *F = S.zF[bt], *Sl = S.zS[bt];
    int* off = S.off[bt];
    const double *pY = Lp.zY[bt], *pF = Lp.zF[bt], *pS = Lp.zS[bt];
    const int* po = Lp.off[bt];
    const int ps = (int)preS, pbz = (int)(totS + preB);
    for (int i = lane; i < nS; i += Team::W) {
      Y[ps + i] = pY[i];
      F[ps + i] = pF[i];
      Sl[ps + i] = pS[i];
    }
    for (int i = lane; i < nB; i += Team::W) {
      Y[pbz + i] = pY[nS + i];
      F[pbz + i] = pF[nS + i];
      Sl[pbz + i] = pS[nS + i];
    }
    for (int k = lane; k < cw; k += Team::W) {
      off[j0 + k] = ps + po[k];
      off[W + j0 + k] = pbz + (po[cw + k] - nS);
    }
    if (c == 0 && lane == 0) off[2 * W] = (int)(totS + totB);
    if ((int)(totS + totB) > R.st.zmax_level) R.st.zmax_level = (int)(totS + totB);
    tm.sync();
    return true;
  }
};

// ------------------------------------------------------------------ one option, nodes split over teams
// A level of the whole-GPU form whose nodes are large next to a share of whole nodes: team
// c of G takes the c-th G-quantile of the level's merged successor points wherever nodes
// begin or end, so one large node is shared by several teams.  What crosses a share boundary:
//   - pass 1: the owner of the segment before the share's first union point (recomputed from
//     that point's successors, own_before);
//   - pass 2: the running minima of h (from the left) and g (from the right) restart at the
//     share's ends and are then combined with the other shares' parts of the same node
//     (phase B, after every team published the minima of its first and last node);
//   - pass 3: the piece at the share's last point ends at the next share's first point, and
//     the first piece needs the slope just left of it; each team publishes its first and last
//     points (phase B) and reads its neighbours' into index -1 and wtot (phase C).
// The w and z points are the ones a single team produces, so the results are the same bits.
struct SplitRec {
  int state;                // A: 0 points of w, 1 empty, 2 overflow
  int first_node, last_node;
  int lhead;                // B: the last point starts its node
  long long cb_last, ca_first;               // A: h minimum of the last node's part, g of the first's
  double fy, ff, fs, ly, lf, ls;             // B: first and last point of w
  long long fgk, fhk, fca, fcb, lgk, lhk, lca, lcb;
};

template <class Team>
struct TcSplit {
  Lay L;  // the shared level banks, the private arrays with w shifted by one point
  TcRun<Team, false, false, true> R;
  int G, c;
  double *zpY, *zpF, *zpS;
  int* poff;
  int capP;
  int n0 = 0, n1 = 0, wtot = 0, ztot = 0, fnode = -1, lnode = -1;

  OB_HD static Lay merge(const Lay& Lp, const GroupLay& S) {
    Lay L = Lp;
    for (int b = 0; b < 2; ++b) {
      L.zY[b] = S.zY[b]; L.zF[b] = S.zF[b]; L.zS[b] = S.zS[b]; L.off[b] = S.off[b];
    }
    L.capZ = S.capZ;
    L.wY += 1; L.wF += 1; L.wS += 1; L.wN += 1;  // index -1 holds the previous share's point
    L.wGK += 1; L.wHK += 1; L.wCA += 1; L.wCB += 1;
    L.capW -= 2;                                 // and index wtot the next share's
    return L;
  }

  OB_HD TcSplit(const Team& tm, const Opt& o, const Lay& Lp, const GroupLay& S, int G_, int c_)
      : L(merge(Lp, S)), R(tm, o, L), G(G_), c(c_), zpY(Lp.zY[0]), zpF(Lp.zF[0]), zpS(Lp.zS[0]),
        poff(Lp.off[0]), capP(Lp.capZ) {}

  // phase A: pass 1 on this team's union points, pass 2 within the share; rec = its record
  OB_HD void phase_a(int t, SplitRec* recs) {
    const Team& tm = R.tm;
    const int lane = tm.lane();
    R.use_banks(t);
    const int nNodes = 2 * (t + 1), W0 = t + 1;
    const long long U = R.ustart_node(t, nNodes);
    const int u0 = (int)(U * c / G), u1 = (int)(U * (c + 1) / G);
    wtot = ztot = 0;
    fnode = lnode = -1;
    int state = 1;
    if (u0 < u1) {
      n0 = R.node_at(t, (long long)u0 + 1) - 1;
      n1 = R.node_at(t, u1);
      // node constants of the share: level t for its nodes, level t+1 for j, j+1
      const int s_lo = n0, s_hi = (n1 < W0 ? n1 : W0) - 1;
      const int b_lo = (n0 > W0 ? n0 : W0) - W0, b_hi = n1 - 1 - W0;
      if (s_lo <= s_hi) {
        R.node_table_range(t, s_lo, s_hi);
        R.node_table_range(t + 1, s_lo, s_hi + 1);
      }
      if (b_lo <= b_hi) {
        R.node_table_range(t, b_lo, b_hi);
        R.node_table_range(t + 1, b_lo, b_hi + 1);
      }
      tm.sync();
      int code = 0;
      if (u0 > R.ustart_node(t, n0) && lane == 0) code = R.own_before(t, n0, u0);
      R.carry0 = tm.bcast0(code);
      R.ub = u0;
      R.ue = u1;
      R.outY = zpY; R.outF = zpF; R.outS = zpS; R.outOff = poff; R.outCap = capP;
      int utot = 0;
      if (!R.pass1(t, wtot, utot, n0, n1)) {
        state = 2;
      } else {
        R.st.upts += utot;
        R.pass2(t, wtot);
        state = wtot > 0 ? 0 : 1;
      }
    }
    if (state == 0) {
      fnode = R.wN()[0];
      lnode = R.wN()[wtot - 1];
    }
    if (lane == 0) {
      SplitRec& r = recs[c];
      r.state = state;
      r.first_node = fnode;
      r.last_node = lnode;
      r.cb_last = state == 0 ? R.wCB()[wtot - 1] : KMAXLL;
      r.ca_first = state == 0 ? R.wCA()[0] : KMAXLL;
    }
    tm.sync();
  }

  // after the barrier: any team's overflow (every team sees the same)
  OB_HD static bool overflow(const SplitRec* recs, int G) {
    for (int g = 0; g < G; ++g)
      if (recs[g].state == 2) return true;
    return false;
  }

  // the nearest team before (dir -1) or after (+1) this one with points of w
  OB_HD int neighbour(const SplitRec* recs, int dir) const {
    for (int g = c + dir; g >= 0 && g < G; g += dir)
      if (recs[g].state == 0) return g;
    return -1;
  }

  // phase B: the running minima of the first and last node combined with the other shares'
  // parts of those nodes; then this team's first and last points into its record
  OB_HD void phase_b(SplitRec* recs) {
    const Team& tm = R.tm;
    const int lane = tm.lane();
    R.lcont = R.rcont = false;
    if (wtot == 0) return;
    long long carryB = KMAXLL, carryA = KMAXLL;
    for (int g = c - 1; g >= 0; --g) {  // h from the left: the earlier parts of the first node
      const SplitRec& r = recs[g];
      if (r.state != 0) continue;
      if (r.last_node != fnode) break;
      R.lcont = true;
      carryB = kmin(carryB, r.cb_last);
      if (r.first_node != r.last_node) break;
    }
    for (int g = c + 1; g < G; ++g) {  // g from the right: the later parts of the last node
      const SplitRec& r = recs[g];
      if (r.state != 0) continue;
      if (r.first_node != lnode) break;
      R.rcont = true;
      carryA = kmin(carryA, r.ca_first);
      if (r.first_node != r.last_node) break;
    }
    long long* CB = R.wCB();
    long long* CA = R.wCA();
    const int* wn = R.wN();
    for (int i = lane; i < wtot; i += Team::W) {
      const int n = wn[i];
      if (n == fnode) CB[i] = kmin(CB[i], carryB);
      if (n == lnode) CA[i] = kmin(CA[i], carryA);
    }
    tm.sync();
    if (lane == 0) {
      SplitRec& r = recs[c];
      const int a = 0, b = wtot - 1;
      r.fy = R.wY()[a]; r.ff = R.wF()[a]; r.fs = R.wS()[a];
      r.fgk = R.wGK()[a]; r.fhk = R.wHK()[a]; r.fca = CA[a]; r.fcb = CB[a];
      r.ly = R.wY()[b]; r.lf = R.wF()[b]; r.ls = R.wS()[b];
      r.lgk = R.wGK()[b]; r.lhk = R.wHK()[b]; r.lca = CA[b]; r.lcb = CB[b];
      r.lhead = (b == 0) ? !R.lcont : (wn[b - 1] != lnode);
    }
    tm.sync();
  }

  // phase C: the neighbours' points at index -1 and wtot, then pass 3; false on overflow
  OB_HD bool phase_c(int t, const SplitRec* recs) {
    const Team& tm = R.tm;
    ztot = 0;
    if (wtot == 0) return true;
    if (R.lcont && tm.lane() == 0) {
      const SplitRec& r = recs[neighbour(recs, -1)];
      R.wY()[-1] = r.ly; R.wF()[-1] = r.lf; R.wS()[-1] = r.ls; R.wN()[-1] = fnode;
      R.wGK()[-1] = r.lgk; R.wHK()[-1] = r.lhk; R.wCA()[-1] = r.lca; R.wCB()[-1] = r.lcb;
    }
    if (R.rcont && tm.lane() == 0) {
      const SplitRec& r = recs[neighbour(recs, 1)];
      R.wY()[wtot] = r.fy; R.wF()[wtot] = r.ff; R.wS()[wtot] = r.fs; R.wN()[wtot] = lnode;
      R.wGK()[wtot] = r.fgk; R.wHK()[wtot] = r.fhk; R.wCA()[wtot] = r.fca; R.wCB()[wtot] = r.fcb;
    }
    tm.sync();
    R.slope0 = 0.0;
    if (R.lcont) {
      R.head_m1 = recs[neighbour(recs, -1)].lhead != 0;
      R.slope0 = R.slope_before(t);
    }
    if (!R.pass3(t, wtot, ztot)) return false;
    R.st.wpts += wtot;
    R.st.zpts += ztot;
    return true;
  }

  // phase D: this team's z points into the shared bank at their prefix, and the offsets of
  // the nodes whose first point is here; cnt[g] = points of team g.  False when the level
  // outgrows the shared bank (every team sees the same).
  OB_HD bool publish(int t, const int* cnt) {
    const Team& tm = R.tm;
    const int lane = tm.lane();
    long long pre = 0, total = 0;
    for (int g = 0; g < G; ++g) {
      if (g < c) pre += cnt[g];
      total += cnt[g];
    }
    if (total > L.capZ) return false;
    const int bt = t & 1;
    double *Y = L.zY[bt], *F = L.zF[bt], *S = L.zS[bt];
    int* off = L.off[bt];
    const int p = (int)pre;
    for (int i = lane; i < ztot; i += Team::W) {
      Y[p + i] = zpY[i];
      F[p + i] = zpF[i];
      S[p + i] = zpS[i];
    }
    if (wtot > 0)
      for (int n = fnode + (R.lcont ? 1 : 0) + lane; n <= lnode; n += Team::W) off[n] = p + poff[n];
    if (c == 0 && lane == 0) off[2 * (t + 1)] = (int)total;
    if ((int)total > R.st.zmax_level) R.st.zmax_level = (int)total;
    tm.sync();
    return true;
  }
};

}  // namespace obk
