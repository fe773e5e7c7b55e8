"""The allocation-free entry point, tt_price_evaluate_static, through the C ABI.

Some callers cannot allocate memory while they price: a quote loop with a
fixed latency budget, a plugin whose host application owns all device memory,
a process whose memory is fixed at start-up.  This entry point serves them
from file-scope arrays instead of a handle.  Here it must reproduce the
handle-based tt_price_evaluate to the FP64 parity tolerance of the other GPU
tests, on two calls in a row (the second call reuses the arrays the first one
left behind), and reject a batch beyond its stated maximum.

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2203_02804_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-6


def _problems():
    rng = np.random.default_rng(4242)
    out = [inputs.two_asset_min_call()]
    for d, n, r, payoff in [(3, 24, 6, "min"), (4, 16, 5, "min"), (2, 32, 8, "max"), (3, 20, 4, "max")]:
        sigma = rng.uniform(0.15, 0.35, d)
        out.append(inputs.Problem(spot=rng.uniform(90, 110, d),
                                  cov=inputs.cov_from(sigma, inputs.equicorrelation(d, 0.3)),
                                  rate=0.02, maturity=1.0, strike=100.0, payoff=payoff,
                                  damping=np.full(d, -1.5), n_grid=n, trunc_L=20.0, max_rank=r,
                                  seed=77 + d + n))
    return out


def test_static_entry_matches_handle_entry_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02804_gb300 import build, ttprice

    build.build()
    lib = ttprice.load_library()
    torch.cuda.set_device(0)
    ps = _problems()
    batch = ttprice.ProblemBatch(ps)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    runs = []
    for _ in range(2):
        prices = (ctypes.c_double * len(ps))()
        diags = (ttprice.tt_diag * len(ps))()
        rc = lib.tt_price_evaluate_static(batch.arr, len(ps), ttprice.TT_FP64, stream, prices, diags)
        assert rc in (ttprice.TT_OK, ttprice.TT_WARN_NOT_CONVERGED), ttprice.status_string(rc)
        assert all(d.status in (ttprice.TT_OK, ttprice.TT_WARN_NOT_CONVERGED) for d in diags)
        runs.append(np.array(prices[:len(ps)]))

    pr = ttprice.Pricer(max_d=4, max_n=64, max_rank=8, max_batch=len(ps), precision="fp64")
    rc, ref, _ = pr.evaluate(ps)
    pr.close()
    assert rc in (ttprice.TT_OK, ttprice.TT_WARN_NOT_CONVERGED)
    for got in runs:
        assert np.all(np.isfinite(got))
        np.testing.assert_array_less(np.abs(got / ref - 1.0), FP64_TOL)

    over = ttprice.TT_STATIC_MAX_BATCH + 1
    prices = (ctypes.c_double * over)()
    rc = lib.tt_price_evaluate_static(batch.arr, over, ttprice.TT_FP64, stream, prices, None)
    assert rc == ttprice.TT_ERR_CAPACITY
