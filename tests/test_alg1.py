"""The paper's parallel scheme (Section 4.2, Algorithm 1) as a CPU comparator, over the
oracle's node steps.  Its partition and synchronisation must not change a single node:

  * prices are bitwise those of the serial oracle for every thread count and block depth,
    for the induction with costs and for the CRR recursion;
  * every node of levels 0..N (0..N-1 for CRR) is computed exactly once;
  * the rounds follow Section 4.2's rules (at least two nodes per thread, fewer threads near
    the root, D = min(L, floor(nodes / p) - 1)), checked against a restatement here and
    against the paper's three-thread example (N = 10, p = 3, L = 3);
  * thread p_0's share matches Section 4.3's estimate of the nodes it processes.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def _rounds_restated(top, p, L):
    """Section 4.2 in words: a round on base level B (B + 1 nodes) first drops threads until
    every thread gets at least two nodes, splits the nodes into blocks of floor((B+1)/p), and
    processes D = min(L, block - 1) levels; the next base level is B - D."""
    out = []
    B = top
    while B > 0:
        while p > 1 and B + 1 < 2 * p:
            p -= 1
        D = min(L, (B + 1) // p - 1)
        out.append((B, D, p))
        B -= D
    return out


@pytest.mark.parametrize("top,p,L", [(11, 3, 3), (1001, 4, 5), (1001, 8, 50), (40, 16, 5),
                                     (7, 1, 3), (2, 2, 1), (300, 5, 1)])
def test_rounds_follow_section_4_2(top, p, L):
    r = oracle.alg1_rounds(top, p, L)
    assert r == _rounds_restated(top, p, L)
    assert r[0][0] == top and sum(D for _, D, _ in r) == top
    for B, D, q in r:
        assert D >= 1 and D <= L
        assert q == 1 or B + 1 >= 2 * q  # at least two nodes per thread
        assert (B + 1) // q >= D + 1     # a block is wider than it is deep
    ps = [q for _, _, q in r]
    assert ps == sorted(ps, reverse=True)


def test_paper_example_three_threads():
    # N = 10, p = 3, L = 3: the leaf level N+1 = 11 has 12 nodes, 4 per thread, so the first
    # round runs D = 3 levels on all three threads; the threads drop to 2 and then 1 as the
    # levels narrow below 2p nodes.
    r = oracle.alg1_rounds(11, 3, 3)
    assert r[0] == (11, 3, 3)
    assert [q for _, _, q in r][-1] == 1
    assert all(B + 1 >= 2 * q for B, _, q in r if q > 1)


CASES = [W.make(k=0.005, N=60), W.make(k=0.01, N=97, payoff=W.CALL),
         W.make(K=95.0, K2=105.0, k=0.01, N=80, payoff=W.SPREAD),
         W.make(k=0.02, N=45, sigma=0.1, payoff=W.CALL), W.make(k=0.0, N=70)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_tc_bitwise_equal_to_serial_oracle(case):
    t = CASES[case]
    N = int(t["N"][0])
    ref, st = oracle.price_ask_bid(t)
    assert st[0] == 0
    for p in (1, 2, 3, 5, 8):
        for L in (1, 2, 5, 50):
            out, rc, per = oracle.alg1_price(t, p, L)
            assert rc == 0
            assert np.array_equal(out.view(np.int64), ref[0].view(np.int64)), (p, L)
            assert per.sum() == (N + 1) * (N + 2) // 2  # levels 0..N, each node once


def test_crr_bitwise_equal_to_serial_oracle():
    for t in (W.appendix_put(500), W.make(k=0.0, N=333, payoff=W.CALL),
              W.make(K=95.0, K2=105.0, k=0.0, N=250, payoff=W.SPREAD)):
        N = int(t["N"][0])
        ref, _ = oracle.crr_price(t)
        for p in (1, 2, 4, 7, 16):
            for L in (1, 5, 50):
                out, rc, per = oracle.alg1_price(t, p, L, crr=True)
                assert rc == 0
                assert np.array_equal(out.view(np.int64), ref.view(np.int64)), (p, L)
                assert per.sum() == N * (N + 1) // 2


def test_thread0_share_matches_section_4_3():
    # Section 4.3: thread p_0 processes about (N+2p+1)(N-2p+4)/(2p) + 4p - 5 nodes of the
    # whole tree, leaves included (exact when every base level splits evenly).
    N, p, L = 1000, 4, 5
    _, rc, per = oracle.alg1_price(W.make(k=0.0, N=N), p, L, crr=False)
    assert rc == 0
    leaves0 = (N + 2) // p
    est = (N + 2 * p + 1) * (N - 2 * p + 4) / (2 * p) + 4 * p - 5
    assert abs(per[0] + leaves0 - est) / est < 0.02
    assert per.sum() == (N + 1) * (N + 2) // 2


def test_error_status_reaches_caller():
    t = W.make(k=0.005, N=50, R=50.0)  # r > u: the model admits arbitrage
    out, rc, _ = oracle.alg1_price(t, 4, 5)
    assert rc == oracle.ERR_ARBITRAGE and np.all(np.isnan(out))
