"""The allocation-free entry point, tt_price_evaluate_static, through the C ABI.

Some callers cannot allocate memory while they price: a quote loop with a
fixed latency budget, a plugin whose host application owns all device memory,
a process whose memory is fixed at start-up.  This entry point serves them
from file-scope arrays instead of a handle.  Here it must reproduce the
handle-based tt_price_evaluate to the parity tolerance of the other GPU tests
(1e-6 in FP64, 1e-4 in the mixed path), on two calls in a row (the second call
reuses the arrays the first one left behind), and reject a batch beyond its
stated maximum.

The result must not depend on what ran before in the process: the kernels'
shared-memory opt-in is process-wide, so the test creates a small pricer and a
large one first, calls the static entry point between them, and then uses both
pricers again.  It passes alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2203_02804_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-6
MIXED_TOL = 1e-4


def _problems():
    rng = np.random.default_rng(4242)
    out = [inputs.two_asset_min_call(max_rank=32)]
    for d, n, r, payoff in [(3, 24, 6, "min"), (4, 16, 5, "min"), (2, 32, 8, "max"), (3, 20, 4, "max")]:
        sigma = rng.uniform(0.15, 0.35, d)
        out.append(inputs.Problem(spot=rng.uniform(90, 110, d),
                                  cov=inputs.cov_from(sigma, inputs.equicorrelation(d, 0.3)),
                                  rate=0.02, maturity=1.0, strike=100.0, payoff=payoff,
                                  damping=np.full(d, -1.5), n_grid=n, trunc_L=20.0, max_rank=r,
                                  seed=77 + d + n))
    return out


def _static(lib, ttprice, batch, n, precision, stream):
    prices = (ctypes.c_double * n)()
    diags = (ttprice.tt_diag * n)()
    rc = lib.tt_price_evaluate_static(batch.arr, n, precision, stream, prices, diags)
    assert rc in (ttprice.TT_OK, ttprice.TT_WARN_NOT_CONVERGED), ttprice.status_string(rc)
    assert all(d.status in (ttprice.TT_OK, ttprice.TT_WARN_NOT_CONVERGED) for d in diags)
    return np.array(prices[:n])


def test_static_entry_matches_handle_entry_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02804_gb300 import build, ttprice

    build.build()
    lib = ttprice.load_library()
    torch.cuda.set_device(0)
    ps = _problems()
    n = len(ps)
    batch = ttprice.ProblemBatch(ps)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    # a small pricer (little shared memory) and a large one (more than the
    # static path's), both created before the first static call
    small = ttprice.Pricer(max_d=4, max_n=64, max_rank=32, max_batch=n, precision="fp64")
    large = ttprice.Pricer(max_d=4, max_n=1024, max_rank=32, max_batch=n, precision="fp64")
    small_mx = ttprice.Pricer(max_d=4, max_n=64, max_rank=32, max_batch=n, precision="mixed", engine="cuda")
    large_mx = ttprice.Pricer(max_d=4, max_n=1024, max_rank=64, max_batch=n, precision="mixed", engine="cuda")
    rc, ref64, _ = small.evaluate(ps)
    assert rc in (ttprice.TT_OK, ttprice.TT_WARN_NOT_CONVERGED)
    rc, refmx, _ = small_mx.evaluate(ps)
    assert rc in (ttprice.TT_OK, ttprice.TT_WARN_NOT_CONVERGED)

    runs64 = [_static(lib, ttprice, batch, n, ttprice.TT_FP64, stream) for _ in range(2)]
    runsmx = [_static(lib, ttprice, batch, n, ttprice.TT_MIXED, stream) for _ in range(2)]
    for got in runs64:
        assert np.all(np.isfinite(got))
        np.testing.assert_array_less(np.abs(got / ref64 - 1.0), FP64_TOL)
    for got in runsmx:
        assert np.all(np.isfinite(got))
        np.testing.assert_array_less(np.abs(got / refmx - 1.0), MIXED_TOL)

    # both pricers still launch after the static calls (the opt-in never fell)
    for pr, ref, tol in ((large, ref64, FP64_TOL), (small, ref64, FP64_TOL), (small_mx, refmx, MIXED_TOL),
                         (large_mx, refmx, MIXED_TOL)):
        rc, again, _ = pr.evaluate(ps)
        assert rc in (ttprice.TT_OK, ttprice.TT_WARN_NOT_CONVERGED), ttprice.status_string(rc)
        np.testing.assert_array_less(np.abs(again / ref - 1.0), tol)
    # a pricer created after the static set-up, smaller than it, then the static path again
    tiny = ttprice.Pricer(max_d=4, max_n=32, max_rank=8, max_batch=n, precision="fp64")
    rc, _, _ = tiny.evaluate(ps[1:])
    assert rc in (ttprice.TT_OK, ttprice.TT_WARN_NOT_CONVERGED), ttprice.status_string(rc)
    got = _static(lib, ttprice, batch, n, ttprice.TT_FP64, stream)
    np.testing.assert_array_less(np.abs(got / ref64 - 1.0), FP64_TOL)
    for pr in (small, large, small_mx, large_mx, tiny):
        pr.close()

    over = ttprice.TT_STATIC_MAX_BATCH + 1
    prices = (ctypes.c_double * over)()
    rc = lib.tt_price_evaluate_static(batch.arr, over, ttprice.TT_FP64, stream, prices, None)
    assert rc == ttprice.TT_ERR_CAPACITY
