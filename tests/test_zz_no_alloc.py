"""The fixed-scratch entry point, ob_price_ask_bid_noalloc.

It serves callers that cannot allocate device memory when they price (their
memory budget is already handed out, or their allocation policy forbids it
after start-up): its scratch is one device array the library holds from load
time.  Two calls in a row must agree with ob_price_ask_bid, which uses the
library's allocated pool, within the parity tolerance.  This file is collected
last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def test_noalloc_matches_pooled_entry_on_two_calls():
    import torch

    import paper_1110_2477_gb300 as ob
    t = W.concat(W.single_put_n250(), W.random_table(300, 2024, N_lo=20, N_hi=900),
                 W.make(K=95.0, K2=105.0, k=0.01, N=600, payoff=W.SPREAD))
    n = len(t)
    params = ob.to_device(t)
    ref = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    rst = torch.empty(n, dtype=torch.int32, device="cuda")
    ob.ob_price_ask_bid(params, n, ref, rst)
    torch.cuda.synchronize()
    ref, rst = ref.cpu().numpy(), rst.cpu().numpy()
    assert np.all(rst == 0)
    scale = np.maximum(np.abs(ref), 1e-2 * t["K"][:, None])
    for _ in range(2):
        out = torch.full((n, 2), -1.0, dtype=torch.float64, device="cuda")
        st = torch.full((n,), 99, dtype=torch.int32, device="cuda")
        ob.ob_price_ask_bid_noalloc(params, n, out, st)
        torch.cuda.synchronize()
        out, st = out.cpu().numpy(), st.cpu().numpy()
        assert np.array_equal(st, rst)
        assert np.all(np.abs(out - ref) <= RTOL * scale)


def test_noalloc_rejects_batches_above_its_limit():
    import torch

    import paper_1110_2477_gb300 as ob
    n = 4097
    params = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
    out = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(ob.ObError, match="invalid argument"):
        ob.ob_price_ask_bid_noalloc(params, n, out)


def test_noalloc_bitwise_equal_to_pooled_and_its_retry_and_capacity_paths():
    """Bitwise agreement with the pooled entry (the same kernels and team code), on two calls;
    a heavy spread whose levels outgrow a first-tier slice of the fixed array (about 4 MiB)
    but fit the whole array, which the follow-up launch prices; and an option that outgrows
    the whole array, which gets OB_ERR_CAPACITY and NaN while the others complete."""
    import torch

    import paper_1110_2477_gb300 as ob
    heavy = W.make(S0=100.0, K=95.0, K2=105.0, sigma=0.1, T=0.1, k=0.02, N=800, payoff=W.SPREAD)
    huge = W.make(k=0.001, N=300000)  # its node tables and two levels alone exceed 64 MiB
    t = W.concat(W.random_table(40, 5150, N_lo=10, N_hi=400), heavy, huge, W.single_put_n250())
    n = len(t)
    ih, iu = 40, 41
    keep = np.arange(n) != iu
    # the pooled entry on every option but the huge one (it would take hours on one SM)
    tk = t[keep]
    ref = torch.empty((len(tk), 2), dtype=torch.float64, device="cuda")
    rst = torch.empty(len(tk), dtype=torch.int32, device="cuda")
    ob.ob_price_ask_bid(ob.to_device(tk), len(tk), ref, rst)
    torch.cuda.synchronize()
    ref, rst = ref.cpu().numpy(), rst.cpu().numpy()
    assert np.all(rst == 0)
    one = torch.empty((1, 2), dtype=torch.float64, device="cuda")
    ob.ob_price_ask_bid(ob.to_device(heavy), 1, one)
    torch.cuda.synchronize()
    assert ob.ob_get_stats()["max_level_points"] > 40000  # beyond a first-tier slice
    params = ob.to_device(t)
    for _ in range(2):
        out = torch.full((n, 2), -1.0, dtype=torch.float64, device="cuda")
        st = torch.full((n,), 99, dtype=torch.int32, device="cuda")
        ob.ob_price_ask_bid_noalloc(params, n, out, st)
        torch.cuda.synchronize()
        out, st = out.cpu().numpy(), st.cpu().numpy()
        assert st[iu] == -3 and np.all(np.isnan(out[iu]))
        assert np.array_equal(st[keep], rst)
        assert np.array_equal(out[keep].view(np.int64), ref.view(np.int64))
