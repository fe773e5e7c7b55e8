"""Warm starts of TT-cross (the learned surrogate's second role): the final pivots
of solved problems (tt_price_pivots) seed the initial right index sets of new
solves (tt_problem.warm_sets), retrieved by the nearest training problem in the
surrogate's standardised feature space (surrogate.PivotMemory).

What the warm start must gain, measured against the cold start on held-out
problems of the surrogate's parameter box (d=5 calls on the minimum, N=128,
rank 32), FP64 path: fewer half-sweeps and fewer integrand evaluations (when
the tests were written: 4.57 -> 3.81 half-sweeps, -13 % evaluations on 256
problems) at equal error against the exact grid sum (oracle/grid_sum.py).
Also: the export/import round trip and the rejection of malformed records."""
import numpy as np
import pytest

from oracle import grid_sum
from paper_2203_02804_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02804_gb300 import build, surrogate, ttprice

    build.build()
    return surrogate, ttprice


def _solve(tp, problems, precision="fp64"):
    pr = tp.Pricer(max_d=5, max_n=128, max_rank=32, max_batch=len(problems), precision=precision, pivot_io=True)
    rc, prices, diags = pr.evaluate(problems)
    recs = [pr.pivots(i) for i in range(len(problems))]
    pr.close()
    return prices, diags, recs


def test_pivot_record_round_trip(env):
    sg, tp = env
    p = inputs.surrogate_batch(1, index=8)[0]
    v0, d0, recs = _solve(tp, [p])
    rec = recs[0]
    # the format: for k = 1..4 a count, then count multi-indices over axes k..4
    off, d = 0, 5
    for k in range(1, d):
        c = int(rec[off])
        assert 1 <= c <= 32
        assert np.all(rec[off + 1:off + 1 + c * (d - k)] < p.n_grid)
        off += 1 + c * (d - k)
    assert off == rec.size
    # the same problem from its own final pivots: as many half-sweeps at most, and a
    # train no further from the exact grid sum.  This option is far out of the money
    # (price 0.56 on spots near 100): both trains carry a few 1e-4 of relative TT error
    # at rank 32 (3e-6 of the spot), so they are compared through the exact sum.
    v1, d1, _ = _solve(tp, [p.with_(warm_sets=rec)])
    assert d1[0].half_sweeps <= d0[0].half_sweeps
    exact = grid_sum.grid_sum_for(p)[0]
    e0, e1 = abs(v0[0] / exact - 1), abs(v1[0] / exact - 1)
    assert e0 < 2e-3 and e1 <= max(1.5 * e0, 1e-5), (e0, e1)


def test_malformed_warm_records_are_refused(env):
    sg, tp = env
    p = inputs.surrogate_batch(1, index=8)[0]
    _, _, recs = _solve(tp, [p])
    bad_index = recs[0].copy()
    bad_index[1] = p.n_grid  # outside the grid
    bad_count = recs[0].copy()
    bad_count[0] = 33  # above the rank cap
    dup = recs[0].copy()
    dup[1 + 4:1 + 8] = dup[1:5]  # bond 1's second multi-index repeats its first
    pr = tp.Pricer(max_d=5, max_n=128, max_rank=32, max_batch=4, precision="fp64", pivot_io=True)
    _, prices, diags = pr.evaluate([p.with_(warm_sets=r) for r in (bad_index, bad_count, dup, recs[0])])
    pr.close()
    assert [d.status for d in diags][:3] == [tp.TT_ERR_INVALID] * 3 and np.all(np.isnan(prices[:3]))
    assert diags[3].status in (tp.TT_OK, tp.TT_WARN_NOT_CONVERGED)
    # without pivot_io a warm start is refused too
    pr = tp.Pricer(max_d=5, max_n=128, max_rank=32, max_batch=1, precision="fp64")
    _, prices, diags = pr.evaluate([p.with_(warm_sets=recs[0])])
    pr.close()
    assert diags[0].status == tp.TT_ERR_INVALID


def test_nearest_training_pivots_save_work_at_equal_error(env):
    sg, tp = env
    train = inputs.surrogate_batch(512, index=5)
    held = inputs.surrogate_batch(128, index=6)
    _, _, trecs = _solve(tp, train)
    f = sg.features(train)
    mem = sg.PivotMemory(train, trecs, (f.mean(0), f.std(0) + 1e-12))
    exact = np.array([grid_sum.grid_sum_for(p)[0] for p in held])
    vc, dc, _ = _solve(tp, held)
    vw, dw, _ = _solve(tp, mem.warm(held))
    hs_c, hs_w = np.mean([d.half_sweeps for d in dc]), np.mean([d.half_sweeps for d in dw])
    ev_c, ev_w = np.mean([d.evaluations for d in dc]), np.mean([d.evaluations for d in dw])
    ec, ew = np.abs(vc / exact - 1), np.abs(vw / exact - 1)
    assert hs_w < hs_c and ev_w < 0.95 * ev_c, (hs_c, hs_w, ev_c, ev_w)
    assert np.median(ew) < 1.5 * np.median(ec) and ew.max() < 2.0 * ec.max(), (np.median(ec), np.median(ew))
