"""Exact-rational restatement of the ask/bid induction -- TEST INFRASTRUCTURE.

The same backward induction as the C++ oracle (Section 3 and Section 4.1 of
Zhang, Roux & Zastawniak: successor max, discount by r, slope restriction to
[-S^a, -S^b], exercise max/min against the expense function of Eq. 1 / Eq. 6,
extra level N+1 with payoff (0,0), no costs at t = 0), carried out in
``fractions.Fraction`` on the exact binary values of the FP64 model constants
u and r.  It gives "the exact result" of the recursion for those inputs, so
the FP64 oracle's rounding error can be measured against it.

It is written independently of the C++ oracle and deliberately differently:
  * collinear breakpoints are removed by an exact slope test;
  * the slope restriction is computed pointwise from its definition,
      v(y) = min( f(y), min_i [ f_i + theta(y_i - y) ] ),
    theta(x) = S^a x (x >= 0), S^b x (x < 0): the infimum over y' of the
    piecewise-linear map y' -> f(y') + theta(y' - y) is attained at y' = y or
    at a breakpoint y_i of f, so v is the lower envelope of f and one cone per
    breakpoint (no sweep).
Only small trees (N up to a few dozen) are practical.
"""
from __future__ import annotations

import math
from fractions import Fraction as Q


class PLQ:
    """Exact piecewise-linear function: breakpoints ys (increasing), values fs, tail slopes."""

    __slots__ = ("ys", "fs", "sL", "sR")

    def __init__(self, ys, fs, sL, sR):
        self.ys, self.fs, self.sL, self.sR = list(ys), list(fs), sL, sR

    def __call__(self, x):
        ys, fs = self.ys, self.fs
        if x <= ys[0]:
            return fs[0] + self.sL * (x - ys[0])
        if x >= ys[-1]:
            return fs[-1] + self.sR * (x - ys[-1])
        lo, hi = 0, len(ys) - 1
        while hi - lo > 1:
            mid = (lo + hi) // 2
            if ys[mid] <= x:
                lo = mid
            else:
                hi = mid
        return fs[lo] + (fs[hi] - fs[lo]) * (x - ys[lo]) / (ys[hi] - ys[lo])

    def simplified(self):
        """Drop breakpoints where the slopes on both sides are exactly equal."""
        ys, fs = self.ys, self.fs
        n = len(ys)
        slopes = [self.sL] + [(fs[i + 1] - fs[i]) / (ys[i + 1] - ys[i]) for i in range(n - 1)] + [self.sR]
        keep = [i for i in range(n) if slopes[i] != slopes[i + 1]]
        if not keep:
            keep = [0]
        return PLQ([ys[i] for i in keep], [fs[i] for i in keep], self.sL, self.sR)


def envelope(F: PLQ, G: PLQ, take_max: bool) -> PLQ:
    """Pointwise max or min: evaluate both at the union of breakpoints and insert every
    strict sign change of F - G (between union points and in the tails)."""
    pick = max if take_max else min
    U = sorted(set(F.ys) | set(G.ys))
    h = [F(y) - G(y) for y in U]
    pts = []
    # left tail crossing
    dl = F.sL - G.sL
    if dl != 0 and h[0] != 0:
        ys = U[0] - h[0] / dl
        if ys < U[0]:
            pts.append(ys)
    for i, y in enumerate(U):
        pts.append(y)
        if i + 1 < len(U) and h[i] * h[i + 1] < 0:
            pts.append(y + (U[i + 1] - y) * h[i] / (h[i] - h[i + 1]))
    dr = F.sR - G.sR
    if dr != 0 and h[-1] != 0:
        ys = U[-1] - h[-1] / dr
        if ys > U[-1]:
            pts.append(ys)
    vals = [pick(F(y), G(y)) for y in pts]
    # tails: compare far-away values
    if take_max:
        sL = min(F.sL, G.sL)
        sR = max(F.sR, G.sR)
    else:
        sL = max(F.sL, G.sL)
        sR = min(F.sR, G.sR)
    return PLQ(pts, vals, sL, sR).simplified()


def restrict(F: PLQ, Sa, Sb) -> PLQ:
    """v(y) = min(f(y), min_i [f_i + theta(y_i - y)]) as an envelope of cones."""
    if F.sR + Sa < 0 or F.sL + Sb > 0:
        raise ValueError("restriction unbounded")
    V = F
    for yi, fi in zip(F.ys, F.fs):
        cone = PLQ([yi], [fi], -Sa, -Sb)  # f_i + Sa (y_i - y) left of y_i, f_i + Sb (y_i - y) right
        V = envelope(V, cone, False)
    return V


def expense(xi, zeta, Sa, Sb, buyer: bool) -> PLQ:
    """Eq. 1 (seller) / Eq. 6 (buyer): one kink, at zeta (seller) or -zeta (buyer)."""
    return PLQ([(-zeta) if buyer else zeta], [(-xi) if buyer else xi], -Sa, -Sb)


def node_step(zu: PLQ, zd: PLQ, r, Sa, Sb, xi, zeta, buyer: bool) -> PLQ:
    w = envelope(zu, zd, True)
    f = PLQ(w.ys, [x / r for x in w.fs], w.sL / r, w.sR / r)
    v = restrict(f, Sa, Sb)
    return envelope(expense(xi, zeta, Sa, Sb, buyer), v, not buyer)


def price(S0, K, K2, sigma, R, T, k, N, payoff, return_functions=False):
    """Exact ask and bid for the FP64 model constants u = exp(sigma sqrt(T/N)), r = exp(R T/N)."""
    dt = T / N
    u = Q(math.exp(sigma * math.sqrt(dt)))
    r = Q(math.exp(R * dt))
    S0q, Kq, K2q, kq = Q(S0), Q(K), Q(K2), Q(k)
    one = Q(1)

    def stock(t, j):
        e = 2 * j - t
        return S0q * (u ** e)

    def pay(S):
        if payoff == 0:
            return Kq, Q(-1)
        if payoff == 1:
            return -Kq, Q(1)
        return max(S - Kq, Q(0)) - max(S - K2q, Q(0)), Q(0)

    zs, zb = [], []
    for j in range(N + 2):
        S = stock(N + 1, j)
        Sa, Sb = (one + kq) * S, (one - kq) * S
        zs.append(expense(Q(0), Q(0), Sa, Sb, False))
        zb.append(expense(Q(0), Q(0), Sa, Sb, True))
    for t in range(N, -1, -1):
        for j in range(t + 1):
            S = stock(t, j)
            kt = Q(0) if t == 0 else kq
            Sa, Sb = (one + kt) * S, (one - kt) * S
            xi, zeta = pay(S)
            zs[j] = node_step(zs[j + 1], zs[j], r, Sa, Sb, xi, zeta, False)
            zb[j] = node_step(zb[j + 1], zb[j], r, Sa, Sb, xi, zeta, True)
    ask, bid = zs[0](Q(0)), -zb[0](Q(0))
    if return_functions:
        return ask, bid, zs[0], zb[0]
    return ask, bid


def price_row(row):
    """Exact (ask, bid) for one record of a workloads table."""
    return price(float(row["S0"]), float(row["K"]), float(row["K2"]), float(row["sigma"]),
                 float(row["R"]), float(row["T"]), float(row["k"]), int(row["N"]),
                 int(row["payoff"]))


def hedge_path(row, moves):
    """Exact hedge along one path (Section 3), for the C++ oracle's hedge_path: at each level t
    of the path each party rebalances from the holding it arrived with (none before t = 0) to
    the y' that attains min over y' of w_t(y')/r + theta_t(y' - y), the rightmost among equal
    minima; the candidates are the breakpoints of w_t and y itself.  The cash of the
    self-financing portfolios that start from the ask and from minus the bid follows
    x_t = r x_{t-1} - theta_t(y_t - y_{t-1}).  The buyer stops at the first level where
    exercising with the holding it arrived with costs less: u_t(y) < v_t(y).
    Returns (ask, bid, hold, cash, stop), hold[t] = (seller, buyer) with None from the stop on."""
    S0, K, K2 = float(row["S0"]), float(row["K"]), float(row["K2"])
    sigma, R, T, k = float(row["sigma"]), float(row["R"]), float(row["T"]), float(row["k"])
    N, payoff = int(row["N"]), int(row["payoff"])
    dt = T / N
    u = Q(math.exp(sigma * math.sqrt(dt)))
    r = Q(math.exp(R * dt))
    S0q, Kq, K2q, kq = Q(S0), Q(K), Q(K2), Q(k)
    one = Q(1)

    def stock(t, j):
        return S0q * (u ** (2 * j - t))

    def pay(S):
        if payoff == 0:
            return Kq, Q(-1)
        if payoff == 1:
            return -Kq, Q(1)
        return max(S - Kq, Q(0)) - max(S - K2q, Q(0)), Q(0)

    jt = [0] * (N + 1)
    for t in range(1, N + 1):
        jt[t] = jt[t - 1] + (1 if moves[t - 1] else 0)
    zs, zb = [], []
    for j in range(N + 2):
        S = stock(N + 1, j)
        Sa, Sb = (one + kq) * S, (one - kq) * S
        zs.append(expense(Q(0), Q(0), Sa, Sb, False))
        zb.append(expense(Q(0), Q(0), Sa, Sb, True))
    F = [None] * (N + 1)  # (seller's w_t / r, buyer's) at the path's node of level t
    for t in range(N, -1, -1):
        for j in range(t + 1):
            S = stock(t, j)
            kt = Q(0) if t == 0 else kq
            Sa, Sb = (one + kt) * S, (one - kt) * S
            xi, zeta = pay(S)
            if j == jt[t]:
                pair = []
                for z in (zs, zb):
                    w = envelope(z[j + 1], z[j], True)
                    pair.append(PLQ(w.ys, [x / r for x in w.fs], w.sL / r, w.sR / r))
                F[t] = pair
            zs[j] = node_step(zs[j + 1], zs[j], r, Sa, Sb, xi, zeta, False)
            zb[j] = node_step(zb[j + 1], zb[j], r, Sa, Sb, xi, zeta, True)
    ask, bid = zs[0](Q(0)), -zb[0](Q(0))

    def rebalance(G, Sa, Sb, y0):
        best = None
        for c in sorted(set(G.ys) | {y0}):
            v = G(c) + (Sa if c >= y0 else Sb) * (c - y0)
            if best is None or v <= best[1]:
                best = (c, v)
        return best

    hold, cash = [], []
    ys, yb, xs, xb = Q(0), Q(0), ask, -bid
    stop = -1
    for t in range(N + 1):
        S = stock(t, jt[t])
        kt = Q(0) if t == 0 else kq
        Sa, Sb = (one + kt) * S, (one - kt) * S
        y, _ = rebalance(F[t][0], Sa, Sb, ys)
        if t > 0:
            xs *= r
        xs -= (Sa if y >= ys else Sb) * (y - ys)
        ys = y
        hb = cb = None
        if stop < 0:
            y, v = rebalance(F[t][1], Sa, Sb, yb)
            xi, zeta = pay(S)
            if expense(xi, zeta, Sa, Sb, True)(yb) < v:
                stop = t
            else:
                if t > 0:
                    xb *= r
                xb -= (Sa if y >= yb else Sb) * (y - yb)
                yb = y
                hb, cb = yb, xb
        hold.append((ys, hb))
        cash.append((xs, cb))
    return ask, bid, hold, cash, stop
