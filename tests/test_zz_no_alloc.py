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
