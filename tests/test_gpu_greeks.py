"""GPU adjoint (ob_greeks) against the oracle's forward-mode dual-number gradient,
against central differences of the GPU prices, and through the autograd.Function.

Gradient tolerance: |g_gpu - g_ref| <= 1e-6 * max(|g_ref|, 1e-3 K).  Prices keep
the parity tolerance of the pricing tests (1e-10 relative, floor 1e-2 K).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

GTOL = 1e-6
NAMES = ("S0", "K", "sigma", "R", "T", "k")


def _ob():
    import paper_1110_2477_gb300 as ob
    return ob


def _gpu_greeks(table):
    import torch
    out, grad, st = _ob().greeks(table)
    torch.cuda.synchronize()
    return out.cpu().numpy(), grad.cpu().numpy(), st.cpu().numpy()


def _check_against_dual(table, nthreads=8):
    out, grad, st = _gpu_greeks(table)
    rout, rgrad, rst = oracle.greeks(table, nthreads=nthreads)
    assert np.array_equal(st, rst)
    K = table["K"]
    scale_v = np.maximum(np.abs(rout), 1e-2 * K[:, None])
    assert np.all(np.abs(out - rout) <= 1e-10 * scale_v)
    scale_g = np.maximum(np.abs(rgrad), 1e-3 * K[:, None, None])
    err = np.abs(grad - rgrad) / scale_g
    worst = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= GTOL, (worst, grad[worst[0]].tolist(), rgrad[worst[0]].tolist())


@pytest.mark.parametrize("seed", range(4))
def test_greeks_match_dual_gradient_small(seed):
    t = W.random_table(24, 8100 + seed, N_lo=1, N_hi=90, k_hi=0.04 if seed % 2 else 0.02)
    t["k"] = np.maximum(t["k"], 1e-4)  # d/dk is one-sided at k = 0
    _check_against_dual(t)


def test_greeks_heavy_cases():
    t = W.concat(W.make(S0=100, K=95, K2=105, sigma=0.1, T=0.1, k=0.02, N=80, payoff=W.SPREAD),
                 W.make(S0=100, K=100, sigma=0.1, T=0.1, k=0.02, N=80, payoff=W.CALL),
                 W.make(K=95, K2=105, k=0.01, N=150, payoff=W.SPREAD),
                 W.single_put_n250()[:1])
    _check_against_dual(t, nthreads=4)


def test_greeks_prices_equal_pricing_entry():
    ob = _ob()
    t = W.random_table(32, 77, N_lo=5, N_hi=300)
    out, _, st = _gpu_greeks(t)
    import torch
    p, ps = ob.price(t)
    torch.cuda.synchronize()
    assert np.array_equal(st, ps.cpu().numpy())
    assert np.array_equal(out.view(np.int64), p.cpu().numpy().view(np.int64))


def test_greeks_central_differences_of_gpu_prices():
    """Central differences (relative bump 1e-5) of the GPU prices; a bump that straddles a
    kink (the 1e-5 and 1e-6 estimates disagree by more than 1e-3) is skipped and counted."""
    ob = _ob()
    import torch
    t = W.random_table(6, 424242, N_lo=30, N_hi=200)
    t["k"] = np.maximum(t["k"], 1e-3)
    out, grad, st = _gpu_greeks(t)
    assert np.all(st == 0)

    def fd(h_rel):
        cols = []
        for a, name in enumerate(NAMES):
            up, dn = t.copy(), t.copy()
            h = h_rel * np.maximum(np.abs(t[name]), 1e-3)
            up[name] = t[name] + h
            dn[name] = t[name] - h
            if name == "K":
                up["K2"] = t["K2"] + h
                dn["K2"] = t["K2"] - h
            pu, _ = ob.price(up)
            pd, _ = ob.price(dn)
            torch.cuda.synchronize()
            cols.append((pu.cpu().numpy() - pd.cpu().numpy()) / (2 * h[:, None]))
        return np.stack(cols, axis=2)

    f5, f6 = fd(1e-5), fd(1e-6)
    scale = np.maximum(np.abs(grad), 1e-3 * t["K"][:, None, None])
    smooth = np.abs(f5 - f6) <= 1e-3 * scale
    assert smooth.sum() >= 0.8 * smooth.size
    assert np.all(np.abs(grad - f5)[smooth] <= 1e-4 * scale[smooth])


def test_autograd_function_contracts_gradient():
    import torch
    ob = _ob()
    t = W.random_table(16, 99, N_lo=20, N_hi=200)
    dev = torch.device("cuda")
    theta = torch.tensor(np.stack([t[n] for n in NAMES], 1), dtype=torch.float64, device=dev,
                         requires_grad=True)
    width = torch.tensor(t["K2"] - t["K"], dtype=torch.float64, device=dev)
    N = torch.tensor(t["N"], device=dev)
    pay = torch.tensor(t["payoff"], device=dev)
    ask, bid, st = ob.ask_bid(theta, width, N, pay)
    wa = torch.linspace(0.5, 1.5, len(t), dtype=torch.float64, device=dev)
    wb = torch.linspace(-1.0, 2.0, len(t), dtype=torch.float64, device=dev)
    (wa * ask + wb * bid).sum().backward()
    _, grad, _ = _gpu_greeks(t)
    want = wa.cpu().numpy()[:, None] * grad[:, 0, :] + wb.cpu().numpy()[:, None] * grad[:, 1, :]
    assert np.all(st.cpu().numpy() == 0)
    np.testing.assert_allclose(theta.grad.cpu().numpy(), want, rtol=1e-13, atol=1e-13)


def test_greeks_config_1024_puts_sampled():
    """The Greeks workload at full size: 1024 puts, N = 1000; the oracle's dual gradient
    checks a sample."""
    t = W.greeks_puts()
    out, grad, st = _gpu_greeks(t)
    assert np.all(st == 0) and np.all(np.isfinite(grad))
    idx = np.array([0, 511, 1023])
    rout, rgrad, _ = oracle.greeks(t[idx], nthreads=3)
    scale_g = np.maximum(np.abs(rgrad), 1e-3 * t["K"][idx][:, None, None])
    assert np.all(np.abs(grad[idx] - rgrad) <= GTOL * scale_g)
    assert np.all(np.abs(out[idx] - rout) <= 1e-10 * np.maximum(np.abs(rout), 1.0))


_MODE_CHILD = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, %(root)r)
import workloads as W, paper_1110_2477_gb300 as ob
t = W.concat(W.random_table(40, 5151, N_lo=2, N_hi=600),
             W.make(k=0.02, N=500, sigma=0.1, payoff=W.CALL),
             W.make(K=95.0, K2=105.0, k=0.015, N=400, sigma=0.12, payoff=W.SPREAD))
out, grad, st = ob.greeks(t)
torch.cuda.synchronize()
np.save(%(npy)r, np.concatenate([out.cpu().numpy().reshape(-1), grad.cpu().numpy().reshape(-1),
                                  st.cpu().numpy().astype(np.float64)]))
"""


def test_full_mode_and_checkpoint_mode_agree(tmp_path):
    """The forward pass that keeps every level's records (the default when they fit) and the
    checkpoint mode with recomputed segments (OB_GREEKS_FULL=0) give the same prices bit for
    bit and the same derivatives up to the order of the atomic additions of the scatter."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = []
    for full in ("1", "0"):
        npy = str(tmp_path / ("g%s.npy" % full))
        env = dict(os.environ, OB_GREEKS_FULL=full)
        r = subprocess.run([sys.executable, "-c", _MODE_CHILD % {"root": root, "npy": npy}], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res.append(np.load(npy))
    n = 42
    a, b = res
    assert np.array_equal(a[-n:], b[-n:]) and np.all(a[-n:] == 0)
    assert np.array_equal(a[:2 * n].view(np.int64), b[:2 * n].view(np.int64))
    ga, gb = a[2 * n:-n], b[2 * n:-n]
    assert np.all(np.abs(ga - gb) <= 1e-11 * np.maximum(np.abs(gb), 1.0))
