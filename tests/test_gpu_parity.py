"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

The oracle (oracle/ttcross.py) runs TT-cross in the paper's order: whole-fiber
elimination for the starting rows and whole-fiber maxvol.  The CUDA kernel
reaches rows of the same quality by its own, cheaper schedule (an elimination
tournament and cyclic block maxvol), so the two build different trains of the
same tensor, and their prices agree to the sum of their TT errors.  Parity is
therefore asserted where the oracle's train has converged: its error against
the exact grid sum (the brute-force full grid at d <= 3, the one-factor grid
sum of oracle/grid_sum.py for equicorrelated min-calls at any d) is stated and
checked in each case, well below the tolerance.  Both sides then run with a
tight stop rule (sweep_tol 1e-10, at most 8 half-sweeps).

Tolerances: 1e-6 relative in FP64, 1e-4 in the mixed path (FP32 fibers and
pivoting, FP64 solve and sums).

Separately, the FP64 kernel is checked against tests/kernel_schedule.py, the
same tensor under the kernel's own schedule in FP64 NumPy: there the pivots
are the same and prices agree to rounding (1e-9), which tests the kernel's
arithmetic apart from its pivot choice.

Sizes span several row blocks, ragged tails, screened fibers (> 512 rows),
ranks up to 40 in FP64; edge cases cover d = 1, full rank, invalid inputs,
the empty batch, batching and graph replay.
"""
import math

import numpy as np
import pytest

import kernel_schedule as ks
from oracle import closed_forms, grid_sum, integrand, ttcross
from paper_2203_02804_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-6
MIXED_TOL = 1e-4
REPLAY_TOL = 1e-9
TIGHT = 1e-10          # stop rule of the converged parity cases (both sides)
# the mixed path's maxvol block product: FP32 on CUDA cores, or 3xTF32 on tensor cores
ENGINES = ["cuda", "tc"]


@pytest.fixture(scope="module")
def tp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02804_gb300 import build, ttprice

    build.build()
    return ttprice


def gpu_price(tp, problems, precision="fp64", **kw):
    max_d = max(p.d for p in problems)
    max_n = max(p.n_grid for p in problems)
    max_r = max(p.max_rank for p in problems)
    pr = tp.Pricer(max_d=max_d, max_n=max_n, max_rank=max_r, max_batch=len(problems),
                   precision=precision, **kw)
    rc, prices, diags = pr.evaluate(problems)
    pr.close()
    return rc, prices, diags


def small_problem(d, n, r, payoff="min", seed=3, rho=0.3, trunc=20.0):
    rng = np.random.default_rng(1000 + 17 * d + n + r)
    spot = rng.uniform(90, 110, d)
    sigma = rng.uniform(0.15, 0.35, d)
    return inputs.Problem(spot=spot, cov=inputs.cov_from(sigma, inputs.equicorrelation(d, rho)),
                          rate=0.02, maturity=1.0, strike=100.0, payoff=payoff,
                          damping=np.full(d, -1.5), n_grid=n, trunc_L=trunc, max_rank=r, seed=seed)


def exact_grid(p):
    """The N^d grid sum the trains approximate."""
    if p.payoff == "min":
        return grid_sum.grid_sum_for(p)[0]
    return integrand.full_grid_price(p)[0]


def oracle_price(p, sweep_tol=TIGHT, theta=1e-8):
    return ttcross.tt_price(p, ttcross.CrossOptions(sweep_tol=sweep_tol, theta=theta))[0]


# converged cases: (d, N, rank, payoff, L); oracle TT error against the exact grid sum
# measured when the cases were chosen: 4e-10 .. 3.6e-7; the kernel's schedule
# (tests/kernel_schedule.py) 1e-9 .. 1.3e-7 on the same cases
CONVERGED = [(2, 64, 32, "min", 40.0), (3, 37, 24, "min", 20.0), (3, 64, 32, "min", 20.0),
             (4, 32, 40, "min", 20.0), (5, 24, 32, "min", 10.0), (5, 32, 40, "min", 20.0),
             (2, 24, 24, "max", 20.0), (2, 64, 32, "max", 20.0), (3, 24, 24, "max", 20.0),
             (3, 32, 32, "max", 20.0)]


def converged_problem(d, n, r, payoff, trunc):
    if d == 2 and payoff == "min":
        return inputs.two_asset_min_call(n_grid=n, max_rank=r)
    return small_problem(d, n, r, payoff=payoff, trunc=trunc)


@pytest.mark.parametrize("d,n,r,payoff,trunc", CONVERGED)
def test_fp64_matches_oracle_on_converged_trains(tp, d, n, r, payoff, trunc):
    p = converged_problem(d, n, r, payoff, trunc)
    exact = exact_grid(p)
    ref = oracle_price(p)
    assert abs(ref / exact - 1) < 5e-7, "the oracle's own train must have converged"
    rc, prices, diags = gpu_price(tp, [p], sweep_tol=TIGHT)
    assert diags[0].status in (tp.TT_OK, tp.TT_WARN_NOT_CONVERGED)
    assert diags[0].terms == (1 if payoff == "min" else d)
    assert abs(prices[0] / ref - 1) < FP64_TOL
    assert abs(prices[0] / exact - 1) < FP64_TOL
    assert abs(diags[0].imag_part) < 1e-6 * abs(prices[0])


@pytest.mark.parametrize("engine", ENGINES)
def test_mixed_matches_oracle_on_converged_trains(tp, engine):
    ps = [converged_problem(*c) for c in CONVERGED if c[2] <= 32]
    _, prices, diags = gpu_price(tp, ps, precision="mixed", engine=engine)
    for p, v, dg in zip(ps, prices, diags):
        assert dg.status in (tp.TT_OK, tp.TT_WARN_NOT_CONVERGED)
        assert abs(v / oracle_price(p) - 1) < MIXED_TOL, (p.d, p.n_grid, p.max_rank, p.payoff)


def test_two_asset_closed_forms_at_fine_grid(tp):
    """N=256 (one fiber of 256 rows x 40 columns): the grid sum is within 1e-11 of
    Stulz (oracle pin); the rank-40 train (TT error ~3e-7) matches the oracle's
    train to 1e-6 and Stulz to 1e-6."""
    for payoff, f in (("min", closed_forms.stulz_min_call), ("max", closed_forms.stulz_max_call)):
        p = inputs.two_asset_min_call(n_grid=256, max_rank=40, payoff=payoff)
        rc, prices, _ = gpu_price(tp, [p], sweep_tol=TIGHT)
        assert abs(prices[0] / oracle_price(p) - 1) < FP64_TOL, payoff
        ref = f(100, 100, 100, 0.01, 1.0, 0.2, 0.3, 0.5)
        assert abs(prices[0] / ref - 1) < FP64_TOL, payoff


def test_single_asset_is_the_grid_sum_and_black_scholes(tp):
    p = inputs.Problem(spot=np.array([105.0]), cov=np.array([[0.0625]]), rate=0.03, maturity=0.8,
                       strike=100.0, payoff="min", damping=np.array([-3.0]), n_grid=512,
                       trunc_L=80.0, max_rank=4, seed=1)
    rc, prices, diags = gpu_price(tp, [p])
    assert rc == tp.TT_OK and diags[0].half_sweeps == 1
    bs = closed_forms.bs_call(105.0, 100.0, 0.03, 0.8, 0.25)
    assert abs(prices[0] / bs - 1) < 1e-10


def test_full_rank_reproduces_full_grid(tp):
    """Rank 16 on a 16x16 grid: the cross interpolates every entry, so the train is
    the full grid sum up to rounding amplified by the pivot blocks' conditioning."""
    p = inputs.two_asset_min_call(n_grid=16, max_rank=16)
    rc, prices, _ = gpu_price(tp, [p])
    exact, _ = integrand.full_grid_price(p)
    assert abs(prices[0] / exact - 1) < 1e-9


def test_benchmark_workload_fp64_and_mixed(tp):
    """d=5, N=128, rank 32 (the benchmark workload), four seeded problems.  At this
    rank the TT error against the exact grid sum is up to ~1.5e-5 for the oracle
    and for the kernel (measured: oracle 2e-7 .. 1.2e-5), so the FP64 path is held
    to the grid sum within 3e-5 and to the oracle within 3e-5, and the mixed path
    to the oracle within 1e-4 (the benchmark's accuracy bar)."""
    ps = inputs.five_asset_batch(4)
    exact = [grid_sum.grid_sum_for(p)[0] for p in ps]
    refs = [oracle_price(p, sweep_tol=1e-6) for p in ps]
    _, p64, d64 = gpu_price(tp, ps, precision="fp64")
    pmx = {e: gpu_price(tp, ps, precision="mixed", engine=e)[1] for e in ENGINES}
    for i in range(len(ps)):
        assert abs(refs[i] / exact[i] - 1) < 3e-5
        assert abs(p64[i] / exact[i] - 1) < 3e-5
        assert abs(p64[i] / refs[i] - 1) < 3e-5
        for e in ENGINES:
            assert abs(pmx[e][i] / refs[i] - 1) < MIXED_TOL, e


# --- the FP64 kernel against its own schedule replayed in FP64 NumPy ---------------

REPLAY_CASES = [(2, 64, 8, "min", 128), (3, 16, 4, "min", 128), (3, 37, 6, "min", 128),
                (4, 13, 5, "min", 128), (3, 50, 8, "min", 64), (3, 50, 16, "min", 128),
                (2, 24, 6, "max", 128), (3, 20, 5, "max", 128)]


@pytest.mark.parametrize("d,n,r,payoff,b", REPLAY_CASES)
def test_fp64_kernel_reproduces_its_schedule(tp, d, n, r, payoff, b):
    """Same pivots, so rounding-level agreement: ragged N, blocks of 64 rows with a
    ragged tail (3 x 50 x 8 = 400 rows), a screened fiber (16 x 50 = 800 rows > 512),
    max-call terms, and the d=2 workload at its rank-8 cap."""
    p = inputs.two_asset_min_call() if (d, n, r) == (2, 64, 8) else small_problem(d, n, r, payoff=payoff)
    rc, prices, _ = gpu_price(tp, [p], block_rows=b)
    ref = ks.replay_price(p, ks.ScheduleOptions(block_rows=b))[0]
    assert abs(prices[0] / ref - 1) < REPLAY_TOL


# --- batching, launch paths and edge cases -------------------------------------------

def test_batch_equals_single_bitwise(tp):
    ps = [small_problem(3, 20, 5, seed=s) for s in range(3)] + [small_problem(2, 24, 6, payoff="max")]
    _, batch, _ = gpu_price(tp, ps)
    for i, p in enumerate(ps):
        _, one, _ = gpu_price(tp, [p])
        assert one[0] == batch[i]


def test_invalid_problems_get_status_and_nan(tp):
    good = small_problem(3, 16, 4)
    bad_pd = good.with_(cov=np.array([[1.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]]))
    bad_strip = good.with_(damping=np.array([-0.2, -0.2, -0.2]))
    bad_sign = good.with_(damping=np.array([0.5, -1.5, -1.5]))
    too_big = good.with_(max_rank=9)
    pr = tp.Pricer(max_d=3, max_n=16, max_rank=8, max_batch=5, precision="fp64")
    rc, prices, diags = pr.evaluate([good, bad_pd, bad_strip, bad_sign, too_big])
    pr.close()
    assert [d.status for d in diags] == [diags[0].status, tp.TT_ERR_NOT_PD, tp.TT_ERR_STRIP,
                                         tp.TT_ERR_STRIP, tp.TT_ERR_CAPACITY]
    assert diags[0].status in (tp.TT_OK, tp.TT_WARN_NOT_CONVERGED)
    assert math.isfinite(prices[0]) and all(math.isnan(v) for v in prices[1:])
    assert rc == tp.TT_ERR_CAPACITY or rc < 0


def test_graph_replay_matches_plain_launches(tp):
    """tt_price_run through a captured CUDA graph (re-captured when the batch layout
    changes, replayed when it repeats) gives the plain launches' prices bitwise."""
    a = [small_problem(3, 16, 4, seed=s) for s in range(3)]
    b = [small_problem(3, 20, 5, seed=s) for s in range(5)]
    out = {}
    for graph in (False, True):
        pr = tp.Pricer(max_d=3, max_n=20, max_rank=5, max_batch=8, precision="mixed", graph=graph)
        got = []
        for batch in (a, b, a, a):
            pr.prepare(batch)
            assert pr.run() == tp.TT_OK
            rc, prices, _ = pr.results()
            got.append(prices)
        pr.close()
        out[graph] = got
    for x, y in zip(out[False], out[True]):
        assert np.array_equal(x, y)
    assert np.array_equal(out[True][0], out[True][2]) and np.array_equal(out[True][2], out[True][3])


def test_empty_batch(tp):
    pr = tp.Pricer(max_d=2, max_n=16, max_rank=4, max_batch=4, precision="fp64")
    rc, prices, diags = pr.evaluate([])
    pr.close()
    assert rc == tp.TT_OK and prices.size == 0


def test_largest_grids_two_assets(tp):
    """The largest grids: N = 2048 in FP64 (one fiber of 2048 rows, screened in
    1024-row blocks) and N = 4096 (the library's largest) in the mixed path.  The
    grid sums equal Stulz to 1e-14 (eta = 0.078); the rank-32 trains are 3e-6
    (oracle) and 7e-6 (the kernel's schedule) from them, the TT error at this rank.
    FP64: the kernel's schedule to rounding and Stulz to 1e-5; mixed: the oracle
    to 1e-4."""
    ref = closed_forms.stulz_min_call(100, 100, 100, 0.01, 1.0, 0.2, 0.3, 0.5)
    p = inputs.two_asset_min_call(n_grid=2048, trunc_L=80.0, max_rank=32)
    rc, prices, diags = gpu_price(tp, [p], sweep_tol=TIGHT)
    assert diags[0].status in (tp.TT_OK, tp.TT_WARN_NOT_CONVERGED)
    assert abs(prices[0] / ks.replay_price(p, ks.ScheduleOptions(sweep_tol=TIGHT))[0] - 1) < REPLAY_TOL
    assert abs(prices[0] / ref - 1) < 1e-5
    q = inputs.two_asset_min_call(n_grid=4096, trunc_L=160.0, max_rank=32)
    for e in ENGINES:
        rc, prices, diags = gpu_price(tp, [q], precision="mixed", engine=e)
        assert diags[0].status in (tp.TT_OK, tp.TT_WARN_NOT_CONVERGED)
        assert abs(prices[0] / oracle_price(q) - 1) < MIXED_TOL, e


def test_mixed_default_rank_tol_at_the_paper_setting(tp):
    """The paper's own setting (N=50, rank cap 15, d = 2, 5, 6): with its default
    rank threshold the mixed single train stays within 1e-4 of the FP64 path."""
    probs = [inputs.paper_table_problem(2 + i % 5).with_(seed=1000 + i, max_rank=15)
             for i in (79, 84, 89, 94, 78, 83, 80, 85)]
    kw = dict(max_d=6, max_n=50, max_rank=15, max_batch=len(probs))
    pr = tp.Pricer(precision="fp64", **kw)
    _, ref, _ = pr.evaluate(probs)
    pr.close()
    pr = tp.Pricer(precision="mixed", **kw)
    _, got, diags = pr.evaluate(probs)
    pr.close()
    assert all(d.status == tp.TT_OK for d in diags)
    assert max(abs(a / b - 1) for a, b in zip(got, ref)) < 1e-4


def test_discretisation_error_estimate(tp):
    """tt_diag.est_discretization_err against the grid's actual error (the exact grid
    sum against the one-factor integral) on the d=5 workload at N = 64, 96, 128 and
    the d=2 workload: within a factor 3 where aliasing dominates, as the
    Poisson-summation model predicts."""
    ps = [inputs.five_asset_batch(1)[0].with_(n_grid=n) for n in (64, 96, 128)]
    ps.append(inputs.two_asset_min_call(n_grid=64, max_rank=32))
    rc, prices, diags = gpu_price(tp, ps, precision="fp64")
    for p, v, dg in zip(ps, prices, diags):
        sig = np.sqrt(np.diag(p.cov))
        rho = float(p.cov[0, 1] / (sig[0] * sig[1]))
        exact = closed_forms.one_factor_price(p.spot, sig, rho, p.strike, p.rate, p.maturity, "min")
        actual = abs(grid_sum.grid_sum_for(p)[0] - exact)
        assert actual / 3 < dg.est_discretization_err < 3 * actual, (p.d, p.n_grid, dg.est_discretization_err, actual)
