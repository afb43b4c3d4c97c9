// ob_adj.cuh -- reverse-mode derivatives of ask and bid with respect to
// (S0, K, sigma, R, T, k): the adjoint of the induction in ob_tc.cuh.
//
// The breakpoint structure is held fixed (the derivative of the piecewise
// linear recursion on the branch the forward pass took).  Levels are swept
// from the root (t = 0) back to the leaves (t = N+1); the adjoint of level t
// needs level t+1's functions and the intermediate arrays of level t, so the
// forward pass keeps level functions at checkpoints every s = ceil(sqrt(N+2))
// levels and each segment between two checkpoints is recomputed once, its levels
// kept, before its adjoint levels run.  In each adjoint level:
//   - passes 1 and 2 are recomputed from level t+1 (pass 2 also records the
//     index at which each running minimum is attained);
//   - pass 3 is rerun in double to record its branch decisions and output
//     positions, then replayed with LD values seeded on the piece's inputs, which
//     yields the local Jacobian of every emitted point; the adjoints of the
//     emitted points are pulled back to the points of w, to the points where the
//     minima of g and h are attained, and to the node constants;
//   - pass 2's g = w + S^a y, h = w + S^b y are pulled back to w;
//   - pass 1 is rerun and its emitted points' adjoints are pulled back to the
//     breakpoints of both successors (level t+1) and to their tail slopes.
// Node constants (S^a lambda, S^b lambda, xi lambda of every node) are chained to
// the six parameters in closed form as they are met.
#pragma once
#include "ob_tc.cuh"

namespace obk {

enum { P_S0 = 0, P_K = 1, P_SIG = 2, P_R = 3, P_T = 4, P_KC = 5, NPAR = 6 };

struct LvRef {
  long long d;  // first double of the level in the store (Y, then F, then S, np each)
  long long o;  // first int of its node offsets
  int np;       // points
};

struct AdjLay {
  double* sd;       // level store: points
  long long sd_cap;
  int* so;          // level store: node offsets
  long long so_cap;
  LvRef* ref;       // [N+2]
  double *zbY[2], *zbF[2], *zbS[2];  // adjoints of two levels' points
  double *wbY, *wbF, *wbS, *wbG, *wbH;
  int *argA, *argB;
  int cap;
};

// Split an arena between the pricing arrays (cap points each), the adjoint arrays
// and the level store.  Returns false if it does not fit.
OB_HD bool carve_greeks(char* base, size_t bytes, int N, int min_cap, Lay& L, AdjLay& A) {
  const size_t nb = node_bytes(N) + 32 * 256 + al256(sizeof(LvRef) * ((size_t)N + 2));
  if (bytes < nb) return false;
  const size_t per = ELEM_BYTES + 11 * sizeof(double) + 2 * sizeof(int);
  size_t cap = (size_t)((double)(bytes - nb) * 0.35) / per;
  if (cap > 0x3fffffff) cap = 0x3fffffff;
  if ((long long)cap < (long long)min_cap) return false;
  char* p = carve_cap(base, N, cap, L);
  auto take = [&](size_t sz) { char* r = p; p += al256(sz); return r; };
  A.ref = (LvRef*)take(sizeof(LvRef) * ((size_t)N + 2));
  for (int b = 0; b < 2; ++b) {
    A.zbY[b] = (double*)take(sizeof(double) * cap);
    A.zbF[b] = (double*)take(sizeof(double) * cap);
    A.zbS[b] = (double*)take(sizeof(double) * cap);
  }
  A.wbY = (double*)take(sizeof(double) * cap);
  A.wbF = (double*)take(sizeof(double) * cap);
  A.wbS = (double*)take(sizeof(double) * cap);
  A.wbG = (double*)take(sizeof(double) * cap);
  A.wbH = (double*)take(sizeof(double) * cap);
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
  A.sd = (double*)p;
  A.sd_cap = (long long)((bytes - (size_t)(p - base)) / sizeof(double)) - 64;
  return A.sd_cap > 0;
}

// Sink of the local-dual replay of a piece: every emitted point's local derivatives are
// contracted with that point's adjoint as soon as the point is produced, in output order
// (left tail, first point if it is part of the output, inside), so no array of LD points
// is kept.
struct PullOut {
  const double *zbY, *zbF, *zbS;
  int w;           // output position of the next emitted point
  int emit_first;  // whether the candidate first point is part of the output
  double adj[LDN];
  double last_slope, tail_slope;
  OB_HD void begin() {}
  OB_HD void pull(const EmT<LD>& em) {
    const double by = zbY[w], bf = zbF[w], bs = zbS[w];
    for (int k = 0; k < LDN; ++k) adj[k] += by * em.y.d[k] + bf * em.f.d[k] + bs * em.s.d[k];
    ++w;
  }
  OB_HD void add_tl(const EmT<LD>& e) { pull(e); }
  OB_HD void set_first(const EmT<LD>& e) {
    if (emit_first) pull(e);
  }
  OB_HD void add_m(const EmT<LD>& e) { pull(e); }
};

OB_HD void atomic_add(double* a, double v) {
#if defined(__CUDA_ARCH__)
  if (v != 0.0) atomicAdd(a, v);
#else
  if (v != 0.0) {  // host builds of this header: compare-and-swap loop
    double old = __atomic_load_n((long long*)a, __ATOMIC_RELAXED) * 0.0 + *a;
    long long expect = dbits(old);
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
  long long sd_top, so_top, seg_sd, seg_so;

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
  OB_HD void pass3_adj(int t, int wtot, const double* zbY, const double* zbF, const double* zbS) {
    const int lane = tm.lane();
    const int W0 = t + 1;
    double carry_slope = 0.0;
    int zpos = 0;
    for (int base = 0; base < wtot; base += Team::W) {
      const int i = base + lane;
      const bool ok = i < wtot;
      PieceIn<double> in;
      PieceOut<double> po;
      po.ntl = po.nm = 0;
      po.first = EmT<double>{0.0, 0.0, 0.0};
      po.last_slope = po.tail_slope = 0.0;
      RecDec rec;
      int node = -1;
      if (ok) {
        R.load_piece(t, i, wtot, in, node);
        piece(in, po, rec);
      }
      double tile_last;
      double prev = tm.prev_last(po.last_slope, carry_slope, tile_last);
      if (ok && in.head) prev = po.tail_slope;
      const int emit_first = (ok && (in.anchor || !same_bits(prev, po.first.s))) ? 1 : 0;
      const int nout = ok ? po.ntl + emit_first + po.nm : 0;
      int total;
      const int p0 = zpos + tm.excl_sum(nout, total);
      if (ok && nout > 0) {
        // seeds: 0 y0, 1 f0, 2 s0, 3 y1, 4 f1, 5 cA0, 6 cA1, 7 cB, 8 Sa, 9 Sb, 10 vu
        PieceIn<LD> li;
        const double vals[11] = {val(in.y0), val(in.f0), val(in.s0), val(in.y1), val(in.f1),
                                 val(in.cA0), val(in.cA1), val(in.cB), val(in.Sa), val(in.Sb), val(in.vu)};
        LD* dst[11] = {&li.y0, &li.f0, &li.s0, &li.y1, &li.f1, &li.cA0, &li.cA1, &li.cB, &li.Sa, &li.Sb, &li.vu};
        for (int k = 0; k < 11; ++k) {
          *dst[k] = mk<LD>(vals[k]);
          dst[k]->d[k] = 1.0;
        }
        li.yu = in.yu; li.head = in.head; li.tail = in.tail; li.seller = in.seller;
        li.anchor = in.anchor; li.Arel = in.Arel; li.Brel = in.Brel;
        PullOut pl;
        pl.zbY = zbY;
        pl.zbF = zbF;
        pl.zbS = zbS;
        pl.w = p0;
        pl.emit_first = emit_first;
        for (int k = 0; k < LDN; ++k) pl.adj[k] = 0.0;
        PlayDec pd{rec.d, 0};
        piece(li, pl, pd);
        const double* adj = pl.adj;
        atomic_add(&A.wbY[i], adj[0]);
        atomic_add(&A.wbF[i], adj[1]);
        atomic_add(&A.wbS[i], adj[2]);
        if (!in.tail) {
          atomic_add(&A.wbY[i + 1], adj[3]);
          atomic_add(&A.wbF[i + 1], adj[4]);
          atomic_add(&A.wbG[A.argA[i + 1]], adj[6]);
        }
        if (in.head) atomic_add(&A.wbG[A.argA[i]], adj[5]);
        atomic_add(&A.wbH[A.argB[i]], adj[7]);
        const int p = node >= W0 ? 1 : 0;
        const int j = node - p * W0;
        acc_node(t, j, p, adj[8], adj[9], in.seller ? adj[10] : -adj[10]);
      }
      carry_slope = tile_last;
      zpos += total;
    }
    tm.sync();
  }

  // ---------------------------------------------------------------- adjoint of pass 2
  OB_HD void pass2_adj(int t, int wtot) {
    const int W0 = t + 1;
    const double* nt = L.nt[t & 1];
    for (int i = tm.lane(); i < wtot; i += Team::W) {
      const double gb = A.wbG[i], hb = A.wbH[i];
      if (gb == 0.0 && hb == 0.0) continue;
      const int n = L.wN[i];
      const int p = n >= W0 ? 1 : 0;
      const int j = n - p * W0;
      const double y = L.wY[i];
      A.wbF[i] += gb + hb;
      A.wbY[i] += nt[4 * j] * gb + nt[4 * j + 1] * hb;
      acc_node(t, j, p, y * gb, y * hb, 0.0);
    }
    tm.sync();
  }

  // ---------------------------------------------------------------- adjoint of pass 1
  OB_HD void pass1_adj(int t, double* zbY, double* zbF, double* zbS) {
    const int lane = tm.lane();
    const int W1 = t + 2, W0 = t + 1, nNodes = 2 * W0;
    const int* o1 = R.inOff;
    const double *Y1 = R.inY, *F1 = R.inF, *S1 = R.inS;
    const double* nt1 = L.nt[(t + 1) & 1];
    const int UB1 = R.ustart(o1, W1, 0, 0, W0);
    const int Utot = R.ustart(o1, W1, UB1, 1, W0);
    int ncur = 0, wpos = 0, carry_own = 0;  // carry_own: 2*own of the last non-duplicate point
    for (int base = 0; base < Utot; base += Team::W) {
      const int q = base + lane;
      const int nl = ncur + lane;
      int nend = 0x7fffffff;
      if (nl < nNodes) {
        const int p = nl >= W0 ? 1 : 0;
        nend = R.ustart(o1, W1, UB1, p, nl - p * W0 + 1);
      }
      int pos, nend_le;
      tm.count_le2(nend, q, base + Team::W, pos, nend_le);
      const int ncur_next = ncur + nend_le;
      P1 e;
      e.dup = true;
      int node = ncur + pos, ql = -1, p = 0, j = 0, aoff = 0, boff = 0, ma = 0, mb = 0;
      if (q < Utot) {
        p = node >= W0 ? 1 : 0;
        j = node - p * W0;
        ql = q - R.ustart(o1, W1, UB1, p, j);
        const int* op = o1 + p * W1;
        aoff = op[j + 1];
        ma = op[j + 2] - aoff;
        boff = op[j];
        mb = aoff - boff;
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
      int cnt = 0;
      int wl = 0;
      bool emit_pt = false;
      if (q < Utot && !e.dup) {
        wl = (ql == 0) ? e.wl_first : v2;
        const double sLw = wl ? e.bL : e.aL, sRw = e.wr ? e.bR : e.aR;
        emit_pt = !same_bits(sLw, sRw);
        cnt = (e.lc ? 1 : 0) + (emit_pt ? 1 : 0) + (e.rc ? 1 : 0);
      }
      int total;
      const int p0 = wpos + tm.excl_sum(cnt, total);
      if (cnt > 0) {
        // sources (seed k -> destination): 0 y; A: 1 value, 2 slope of the evaluated piece,
        // 3 its anchor y, 4 left slope, 5 right slope; B: 6..10 alike
        const double* Ay = Y1 + aoff; const double* Af = F1 + aoff; const double* As = S1 + aoff;
        const double* By = Y1 + boff; const double* Bf = F1 + boff; const double* Bs = S1 + boff;
        const double aTL = -nt1[4 * (j + 1)], bTL = -nt1[4 * j];
        // destination encoding: >= 0: (array id 0 y / 1 f / 2 s) * 2^28 + index in level t+1;
        // -1: A's tail slope, -2: B's tail slope, -3: none
        long long dstk[11];
        LD sy = mk<LD>(e.y);
        sy.d[0] = 1.0;
        dstk[0] = e.fromA ? (0LL << 28) + aoff + e.ia : (0LL << 28) + boff + e.ib;
        auto side = [&](const double* Yv, const double* Fv, const double* Sv, int off, bool bp, int ib_,
                        int kb_, double TL, int tailcode, int s0, LD& val_, LD& sl, LD& sr) {
          long long* d = dstk + s0;
          if (bp) {
            val_ = mk<LD>(Fv[ib_]); val_.d[s0] = 1.0; d[0] = (1LL << 28) + off + ib_;
            d[1] = -3; d[2] = -3;
            sl = mk<LD>(ib_ > 0 ? Sv[ib_ - 1] : TL); sl.d[s0 + 3] = 1.0;
            d[3] = ib_ > 0 ? (2LL << 28) + off + ib_ - 1 : tailcode;
            sr = mk<LD>(Sv[ib_]); sr.d[s0 + 4] = 1.0; d[4] = (2LL << 28) + off + ib_;
          } else {
            const int a0 = kb_ >= 0 ? kb_ : 0;
            LD f = mk<LD>(Fv[a0]); f.d[s0] = 1.0; d[0] = (1LL << 28) + off + a0;
            LD s = mk<LD>(kb_ >= 0 ? Sv[kb_] : TL); s.d[s0 + 1] = 1.0;
            d[1] = kb_ >= 0 ? (2LL << 28) + off + kb_ : tailcode;
            LD ya = mk<LD>(Yv[a0]); ya.d[s0 + 2] = 1.0; d[2] = (0LL << 28) + off + a0;
            val_ = f + s * (sy - ya);
            sl = mk<LD>(val(s)); sl.d[s0 + 3] = 1.0; d[3] = d[1];
            sr = mk<LD>(val(s)); sr.d[s0 + 4] = 1.0; d[4] = d[1];
          }
        };
        LD a, aL, aR, b, bL, bR;
        side(Ay, Af, As, aoff, e.aBp, e.ia, e.ka, aTL, -1, 1, a, aL, aR);
        side(By, Bf, Bs, boff, e.bBp, e.ib, e.kb, bTL, -2, 6, b, bL, bR);
        double adj[11];
        for (int k = 0; k < 11; ++k) adj[k] = 0.0;
        int w = p0;
        auto pull = [&](const LD& ey, const LD& ef, const LD& es) {
          const double by = A.wbY[w], bf = A.wbF[w], bs = A.wbS[w];
          for (int k = 0; k < 11; ++k) adj[k] += by * ey.d[k] + bf * ef.d[k] + bs * es.d[k];
          ++w;
        };
        if (e.lc) {
          const int W_ = e.lc_w;
          const LD vW = W_ ? b : a, vO = W_ ? a : b, sW = W_ ? bL : aL, sO = W_ ? aL : bL;
          const LD x = sy + (vW - vO) / (sO - sW);
          pull(x, vW + sW * (x - sy), sW);
        }
        if (emit_pt) {
          const bool pickA = okey(e.a) >= okey(e.b);
          pull(sy, pickA ? a : b, e.wr ? bR : aR);
        }
        if (e.rc) {
          const int W_ = e.rc_w;
          const LD vW = W_ ? b : a, vO = W_ ? a : b, sW = W_ ? bR : aR, sO = W_ ? aR : bR;
          const LD x = sy + (vW - vO) / (sO - sW);
          pull(x, vW + sW * (x - sy), sO);
        }
        for (int k = 0; k < 11; ++k) {
          if (adj[k] == 0.0) continue;
          const long long d = dstk[k];
          if (d == -3) continue;
          if (d == -1) { acc_node(t + 1, j + 1, p, -adj[k], 0.0, 0.0); continue; }
          if (d == -2) { acc_node(t + 1, j, p, -adj[k], 0.0, 0.0); continue; }
          const int arr = (int)(d >> 28), idx = (int)(d & ((1LL << 28) - 1));
          atomic_add(arr == 0 ? &zbY[idx] : (arr == 1 ? &zbF[idx] : &zbS[idx]), adj[k]);
        }
      }
      wpos += total;
      ncur = ncur_next;
    }
    tm.sync();
  }

  OB_HD void zero(double* a, int n) {
    for (int i = tm.lane(); i < n; i += Team::W) a[i] = 0.0;
  }

  // ---------------------------------------------------------------- driver
  // Returns a status; on success lane 0's gA / gB hold d ask / d theta and d bid / d theta.
  OB_HD int run(double& ask, double& bid, double* gA, double* gB) {
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
    // forward, keeping checkpoints
    for (int t = N; t >= 0; --t) {
      const int b1 = (t + 1) & 1;
      R.inY = L.zY[b1]; R.inF = L.zF[b1]; R.inS = L.zS[b1]; R.inOff = L.off[b1];
      if (!level_to_bank(t)) return ST_CAPACITY;
      if (is_ckpt(t) && !store_from_bank(t)) return ST_CAPACITY;
    }
    const long long ckpt_sd = sd_top, ckpt_so = so_top;
    // reverse sweep, one segment per checkpoint, from the root upward
    int cur = 0;  // adjoint bank of the current level
    int lo = 0;   // lowest level whose functions the next segment must provide
    bool seeded = false;
    for (int c = 0; c <= N + 1; ++c) {
      if (!is_ckpt(c)) continue;
      if (c < lo) continue;
      // recompute levels c-1 .. lo from the checkpoint c (kept in the store after the checkpoints)
      sd_top = ckpt_sd;
      so_top = ckpt_so;
      for (int t = c - 1; t >= lo; --t) {
        in_from_store(t + 1);
        if (!level_to_bank(t) || !store_from_bank(t)) return ST_CAPACITY;
      }
      if (!seeded && c > 0) {  // root: seed the adjoints of level 0
        seeded = true;
        const LvRef r0 = A.ref[0];
        const double* Y0 = A.sd + r0.d;
        const double* F0 = Y0 + r0.np;
        const double* S0v = F0 + r0.np;
        const int* off0 = A.so + r0.o;
        zero(A.zbY[cur], r0.np); zero(A.zbF[cur], r0.np); zero(A.zbS[cur], r0.np);
        tm.sync();
        const double lam0 = L.lam[0];
        double vals[2];
        for (int p = 0; p < 2; ++p) {
          const int b = off0[p], e = off0[p + 1];
          const double sc = (p == 0 ? 1.0 : -1.0) / lam0;
          const double tailL = -L.nt[0][0];
          double v;
          if (e <= b) { vals[p] = 0.0; continue; }
          if (!klt(Y0[b], 0.0)) {
            v = F0[b] + tailL * (0.0 - Y0[b]);
            if (lane == 0) { A.zbF[cur][b] += sc; A.zbY[cur][b] += sc * (-tailL); }
            acc_node(0, 0, p, lane == 0 ? sc * Y0[b] : 0.0, 0.0, 0.0);
          } else {
            int k = b;
            while (k + 1 < e && kle(Y0[k + 1], 0.0)) ++k;
            v = F0[k] + S0v[k] * (0.0 - Y0[k]);
            if (lane == 0) { A.zbF[cur][k] += sc; A.zbS[cur][k] += sc * (-Y0[k]); A.zbY[cur][k] += sc * (-S0v[k]); }
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
      // adjoint levels lo .. c-1 (each needs level t+1 <= c)
      for (int t = lo; t <= c - 1; ++t) {
        in_from_store(t + 1);
        R.node_table(t + 1);
        R.node_table(t);
        tm.sync();
        int wtot, utot;
        if (!R.pass1(t, wtot, utot)) return ST_CAPACITY;
        if (wtot > A.cap) return ST_CAPACITY;
        R.template pass2<true>(t, wtot, A.argA, A.argB);
        zero(A.wbY, wtot); zero(A.wbF, wtot); zero(A.wbS, wtot); zero(A.wbG, wtot); zero(A.wbH, wtot);
        tm.sync();
        pass3_adj(t, wtot, A.zbY[cur], A.zbF[cur], A.zbS[cur]);
        pass2_adj(t, wtot);
        const int nxt = cur ^ 1;
        const int np1 = A.ref[t + 1].np;
        if (np1 > A.cap) return ST_CAPACITY;
        zero(A.zbY[nxt], np1); zero(A.zbF[nxt], np1); zero(A.zbS[nxt], np1);
        tm.sync();
        pass1_adj(t, A.zbY[nxt], A.zbF[nxt], A.zbS[nxt]);
        cur = nxt;
      }
      lo = c;
    }
    // leaves: only their slopes -S^b_{N+1,j} depend on the parameters
    {
      const LvRef rl = A.ref[N + 1];
      const int W = N + 2;
      for (int n = lane; n < rl.np; n += Team::W) {
        const int p = n >= W ? 1 : 0;
        const int j = n - p * W;
        acc_node(N + 1, j, p, 0.0, -A.zbS[cur][n], 0.0);
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
