"""Brute-force hedging programs on the non-recombining tree -- TEST INFRASTRUCTURE.

An independent formulation of the ask and bid prices of Section 3 (Zhang,
Roux & Zastawniak) that never builds a piecewise-linear function: the prices
are computed directly from their financial definitions as linear programs on
the full binary (non-recombining) tree of depth N+1, with the model of
Section 4.1 (u = exp(sigma sqrt(T/N)), r = exp(R T/N), extra instant N+1 with
payoff (0,0), no transaction costs at t = 0, S^a = (1+k)S, S^b = (1-k)S).

Ask (seller's superhedging price, Section 3): the least initial cash x_0
(with no stock) from which a self-financing strategy covers delivery of the
payoff portfolio (xi_t, zeta_t) at every node, whenever the buyer exercises.
At a node with incoming holding (c, y) -- cash already grown by r -- the
seller must be able to deliver: c >= u_t(y) of Eq. 1; then rebalances
y -> y + b - s paying S^a b and receiving S^b s.

Bid (buyer's price, Section 3): the largest amount beta the buyer can borrow
at t = 0 against the option: over all stopping times tau (exercise nodes, at
most one on every path; a path not stopped by N stops at N+1 with payoff
(0,0)) and self-financing strategies started from (-beta, 0), the incoming
holding at tau must satisfy c >= u'_tau(y) of Eq. 6.  Stopping times are
enumerated exhaustively for N <= 3; for larger N a mixed-integer program
chooses tau and a final linear program with that tau fixed gives the value.

The expense functions are convex and piecewise linear with two pieces
(slopes -S^a left of the kink, -S^b right of it), so "c >= u(y)" is two
linear inequalities.  Only tiny trees (N <= 6) are practical.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy.optimize import linprog, milp, LinearConstraint, Bounds

_LP_OPTS = {"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10}


class _Tree:
    """Nodes of the non-recombining tree, levels 0..N (decision nodes) and N+1 (leaves)."""

    def __init__(self, S0, K, K2, sigma, R, T, k, N, payoff):
        self.N = N
        dt = T / N
        self.u = math.exp(sigma * math.sqrt(dt))
        self.r = math.exp(R * dt)
        self.S0, self.K, self.K2, self.k, self.payoff = S0, K, K2, k, payoff
        # node id -> (level, number of up moves, parent id or -1)
        self.nodes = [(0, 0, -1)]
        self.children = {}
        level = [0]
        for t in range(1, N + 2):
            nxt = []
            for p in level:
                ups = self.nodes[p][1]
                kids = []
                for up in (1, 0):
                    self.nodes.append((t, ups + up, p))
                    kids.append(len(self.nodes) - 1)
                self.children[p] = kids
                nxt.extend(kids)
            level = nxt

    def stock(self, n):
        t, ups, _ = self.nodes[n]
        return self.S0 * self.u ** (2 * ups - t)

    def bid_ask_stock(self, n):
        t = self.nodes[n][0]
        S = self.stock(n)
        kt = 0.0 if t == 0 else self.k
        return (1 + kt) * S, (1 - kt) * S

    def payoff_at(self, n):
        """(xi, zeta) delivered on exercise at node n; (0, 0) at the extra instant N+1."""
        t = self.nodes[n][0]
        if t == self.N + 1:
            return 0.0, 0.0
        S = self.stock(n)
        if self.payoff == 0:
            return self.K, -1.0
        if self.payoff == 1:
            return -self.K, 1.0
        return max(S - self.K, 0.0) - max(S - self.K2, 0.0), 0.0


def _expense_rows(Sa, Sb, xi, zeta, buyer):
    """The two lines whose max is u(y) (Eq. 1 seller, Eq. 6 buyer): list of (a, b) with u >= a + b y."""
    if buyer:
        # u'(y) = -xi + (y + zeta)^- Sa - (y + zeta)^+ Sb = -xi + max(-Sa (y+zeta), -Sb (y+zeta))
        return [(-xi - Sa * zeta, -Sa), (-xi - Sb * zeta, -Sb)]
    # u(y) = xi + max(-Sa (y - zeta), -Sb (y - zeta))
    return [(xi + Sa * zeta, -Sa), (xi + Sb * zeta, -Sb)]


class _LP:
    """Tiny sparse LP builder: variables by name, rows as dicts."""

    def __init__(self):
        self.names = {}
        self.lb, self.ub = [], []
        self.ub_rows, self.ub_rhs = [], []
        self.eq_rows, self.eq_rhs = [], []
        self.integ = []

    def var(self, name, lo=-np.inf, hi=np.inf, integer=False):
        self.names[name] = len(self.lb)
        self.lb.append(lo)
        self.ub.append(hi)
        self.integ.append(1 if integer else 0)
        return self.names[name]

    def le(self, coefs, rhs):
        self.ub_rows.append(coefs)
        self.ub_rhs.append(rhs)

    def eq(self, coefs, rhs):
        self.eq_rows.append(coefs)
        self.eq_rhs.append(rhs)

    def dense(self, rows):
        A = np.zeros((len(rows), len(self.lb)))
        for i, row in enumerate(rows):
            for j, v in row.items():
                A[i, j] += v
        return A


def _incoming(tr, n, lp, x0):
    """(cash coefficient dict, stock coefficient dict) of the holding entering node n."""
    p = tr.nodes[n][2]
    if p < 0:
        return {x0: 1.0}, {}
    return {lp.names[("x", p)]: tr.r}, {lp.names[("y", p)]: 1.0}


def _add(d, e, scale=1.0):
    out = dict(d)
    for k, v in e.items():
        out[k] = out.get(k, 0.0) + scale * v
    return out


def ask(S0, K, K2, sigma, R, T, k, N, payoff):
    """Seller's superhedging price by one linear program."""
    tr = _Tree(S0, K, K2, sigma, R, T, k, N, payoff)
    lp = _LP()
    x0 = lp.var("x0")
    for n, (t, _, _) in enumerate(tr.nodes):
        if t <= N:
            lp.var(("x", n)); lp.var(("y", n))
            lp.var(("b", n), 0.0); lp.var(("s", n), 0.0)
    for n, (t, _, _) in enumerate(tr.nodes):
        Sa, Sb = tr.bid_ask_stock(n)
        xi, zeta = tr.payoff_at(n)
        cin, yin = _incoming(tr, n, lp, x0)
        # cover exercise (or expiry at N+1): c_in >= a + b y_in  <=>  -c_in + b y_in <= -a
        for a, b in _expense_rows(Sa, Sb, xi, zeta, buyer=False):
            lp.le(_add({k_: -v for k_, v in cin.items()}, yin, b), -a)
        if t <= N:
            xv, yv, bv, sv = (lp.names[(c, n)] for c in "xybs")
            # y = y_in + b - s ; x <= c_in - Sa b + Sb s
            lp.eq(_add({yv: 1.0, bv: -1.0, sv: 1.0}, yin, -1.0), 0.0)
            lp.le(_add({xv: 1.0, bv: Sa, sv: -Sb}, cin, -1.0), 0.0)
    c = np.zeros(len(lp.lb))
    c[x0] = 1.0
    res = linprog(c, A_ub=lp.dense(lp.ub_rows), b_ub=lp.ub_rhs, A_eq=lp.dense(lp.eq_rows),
                  b_eq=lp.eq_rhs, bounds=list(zip(lp.lb, lp.ub)), method="highs-ds",
                  options=_LP_OPTS)
    if res.status != 0:
        raise RuntimeError("seller LP failed: %s" % res.message)
    return float(res.fun)


def _stopping_times(tr, n):
    """All stopping times of the subtree at n, as frozensets of stop nodes."""
    t = tr.nodes[n][0]
    if t == tr.N + 1:
        return [frozenset([n])]
    out = [frozenset([n])]
    a, b = tr.children[n]
    for sa in _stopping_times(tr, a):
        for sb in _stopping_times(tr, b):
            out.append(sa | sb)
    return out


def _buyer_lp(tr, stops):
    """max beta for a fixed stopping time (set of stop nodes)."""
    lp = _LP()
    beta = lp.var("beta")
    x0 = lp.var("x0")
    lp.eq({x0: 1.0, beta: 1.0}, 0.0)  # initial cash is -beta
    alive = set()  # decision nodes strictly before the stop on their path

    def walk(n):
        if n in stops:
            return
        alive.add(n)
        for c in tr.children[n]:
            walk(c)

    walk(0)
    for n in sorted(alive):
        lp.var(("x", n)); lp.var(("y", n)); lp.var(("b", n), 0.0); lp.var(("s", n), 0.0)
    for n in sorted(alive):
        Sa, Sb = tr.bid_ask_stock(n)
        cin, yin = _incoming(tr, n, lp, x0)
        xv, yv, bv, sv = (lp.names[(c, n)] for c in "xybs")
        lp.eq(_add({yv: 1.0, bv: -1.0, sv: 1.0}, yin, -1.0), 0.0)
        lp.le(_add({xv: 1.0, bv: Sa, sv: -Sb}, cin, -1.0), 0.0)
    for n in stops:
        Sa, Sb = tr.bid_ask_stock(n)
        xi, zeta = tr.payoff_at(n)
        cin, yin = _incoming(tr, n, lp, x0)
        for a, b in _expense_rows(Sa, Sb, xi, zeta, buyer=True):
            lp.le(_add({k_: -v for k_, v in cin.items()}, yin, b), -a)
    c = np.zeros(len(lp.lb))
    c[beta] = -1.0
    res = linprog(c, A_ub=lp.dense(lp.ub_rows), b_ub=lp.ub_rhs, A_eq=lp.dense(lp.eq_rows),
                  b_eq=lp.eq_rhs, bounds=list(zip(lp.lb, lp.ub)), method="highs-ds",
                  options=_LP_OPTS)
    if res.status == 2:  # infeasible stopping time cannot happen (solvency is reachable) but be safe
        return -np.inf
    if res.status != 0:
        raise RuntimeError("buyer LP failed: %s" % res.message)
    return -float(res.fun)


def bid_enumerate(S0, K, K2, sigma, R, T, k, N, payoff):
    """Buyer's price by enumerating every stopping time (N <= 3)."""
    tr = _Tree(S0, K, K2, sigma, R, T, k, N, payoff)
    if N > 3:
        raise ValueError("enumeration is only practical for N <= 3")
    return max(_buyer_lp(tr, s) for s in _stopping_times(tr, 0))


def bid_milp(S0, K, K2, sigma, R, T, k, N, payoff, ybound=10.0, xbound=1e4):
    """Buyer's price: a mixed-integer program picks the stopping time (binary stop
    indicators with big-M solvency rows); the value is then re-solved exactly by
    the linear program for that stopping time."""
    tr = _Tree(S0, K, K2, sigma, R, T, k, N, payoff)
    lp = _LP()
    beta = lp.var("beta", -xbound, xbound)
    x0 = lp.var("x0", -xbound, xbound)
    lp.eq({x0: 1.0, beta: 1.0}, 0.0)
    dec = [n for n, nd in enumerate(tr.nodes) if nd[0] <= N]
    for n in dec:
        lp.var(("x", n), -xbound, xbound); lp.var(("y", n), -ybound, ybound)
        lp.var(("b", n), 0.0, 2 * ybound); lp.var(("s", n), 0.0, 2 * ybound)
        lp.var(("d", n), 0.0, 1.0, integer=True)

    def anc(n):  # proper ancestors
        out = []
        p = tr.nodes[n][2]
        while p >= 0:
            out.append(p)
            p = tr.nodes[p][2]
        return out

    Smax = max(tr.bid_ask_stock(n)[0] for n in range(len(tr.nodes)))
    M = 2 * xbound * max(tr.r, 1.0) + Smax * (ybound + 2) + 4 * (K2 + K) + 10.0
    for n, (t, _, _) in enumerate(tr.nodes):
        Sa, Sb = tr.bid_ask_stock(n)
        cin, yin = _incoming(tr, n, lp, x0)
        # alive_n = 1 - sum_{proper ancestors} d_a ; stop_n = d_n (t <= N) or alive_n (t = N+1)
        dsum = {lp.names[("d", a)]: 1.0 for a in anc(n)}
        if t <= N:
            dn = lp.names[("d", n)]
            lp.le(_add({dn: 1.0}, dsum), 1.0)  # d_n <= alive_n
            xv, yv, bv, sv = (lp.names[(c, n)] for c in "xybs")
            lp.eq(_add({yv: 1.0, bv: -1.0, sv: 1.0}, yin, -1.0), 0.0)
            lp.le(_add({xv: 1.0, bv: Sa, sv: -Sb}, cin, -1.0), 0.0)
            stop = {dn: 1.0}
            stop_const = 0.0
        else:
            stop = {k_: -1.0 for k_ in dsum}  # alive = 1 - sum
            stop_const = 1.0
        xi, zeta = tr.payoff_at(n)
        for a, b in _expense_rows(Sa, Sb, xi, zeta, buyer=True):
            # a + b y_in - c_in <= M (1 - stop)
            row = _add({k_: -v for k_, v in cin.items()}, yin, b)
            row = _add(row, stop, M)
            lp.le(row, -a + M * (1.0 - stop_const))
    nv = len(lp.lb)
    c = np.zeros(nv)
    c[beta] = -1.0
    cons = []
    if lp.ub_rows:
        cons.append(LinearConstraint(lp.dense(lp.ub_rows), -np.inf, np.asarray(lp.ub_rhs)))
    if lp.eq_rows:
        r = np.asarray(lp.eq_rhs)
        cons.append(LinearConstraint(lp.dense(lp.eq_rows), r, r))
    res = milp(c, constraints=cons, integrality=np.asarray(lp.integ),
               bounds=Bounds(np.asarray(lp.lb), np.asarray(lp.ub)),
               options={"mip_rel_gap": 1e-12, "presolve": True})
    if res.status != 0:
        raise RuntimeError("buyer MILP failed: %s" % res.message)
    # recover the stopping time and re-solve its LP exactly
    stops = set()

    def walk(n):
        t = tr.nodes[n][0]
        if t == N + 1 or res.x[lp.names[("d", n)]] > 0.5:
            stops.add(n)
            return
        for ch in tr.children[n]:
            walk(ch)

    walk(0)
    return _buyer_lp(tr, frozenset(stops))


def price_row(row, bid_method="auto"):
    """(ask, bid) for one record of a workloads table."""
    args = (float(row["S0"]), float(row["K"]), float(row["K2"]), float(row["sigma"]),
            float(row["R"]), float(row["T"]), float(row["k"]), int(row["N"]), int(row["payoff"]))
    a = ask(*args)
    N = args[7]
    if bid_method == "enumerate" or (bid_method == "auto" and N <= 2):
        b = bid_enumerate(*args)
    else:
        b = bid_milp(*args)
    return a, b
