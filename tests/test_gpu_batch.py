"""The heterogeneous batch at full size: 4096 problems of uneven d, N and rank,
calls on the minimum and on the maximum mixed 50/50, in one launch.

The whole batch runs in the launch configuration the library uses for any batch.
Every price is checked for the properties that hold at any size: a finite
positive price, a status that is OK or not-converged, and an imaginary part of
the grid sum that is small next to the price (the midpoint grid is symmetric, so
the exact grid sum is real and the imaginary part is TT error).  Many draws cap
the rank below what the integrand needs (rank 8 at d = 10); their sweeps end
unconverged with a TT error of up to tens of percent in either precision, so the
tight bound on the imaginary part applies to converged problems and the loose
one only rules out a blow-up.

Parity is checked element by element on a stratified sample: one problem per
(d, N, payoff) cell whose FP64 oracle train has converged, with the oracle's
prices stored in tests/golden/hetero_stratified.json by
tests/golden/make_hetero_golden.py (which calls only the oracle).  First-tier
cells (oracle within 1e-7 of the exact grid sum, or, for the call on the
maximum, every term's stop rule held with an imaginary part below 1e-7) are
held to 1e-6 in FP64 and 1e-4 in the mixed path; second-tier cells (error
measure below 1e-5) to 1e-4 in the mixed path.  The mixed bound carries the
FP32 floor of 2e-7 times the spot: the integrand's terms are of the spot's size,
so single-precision sums leave that much absolute error on prices far below it."""
import json
import math
import os

import numpy as np
import pytest

from paper_2203_02804_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hetero_stratified.json")


@pytest.fixture(scope="module")
def tp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02804_gb300 import build, ttprice

    build.build()
    return ttprice


def _cost(p):
    return p.d * p.n_grid * p.max_rank ** 2 * (p.d if p.payoff == "max" else 1)


@pytest.fixture(scope="module")
def batch():
    return inputs.mixed_batch(4096)


def _run(tp, problems, precision, engine="auto"):
    pr = tp.Pricer(max_d=10, max_n=256, max_rank=32, max_batch=len(problems), precision=precision,
                   engine=engine)
    rc, prices, diags = pr.evaluate(problems)
    pr.close()
    return rc, prices, diags


def _golden():
    with open(GOLDEN) as f:
        g = json.load(f)
    return g["cells"], g.get("cells_tier2", [])


def _mixed_ok(price, ref, p):
    return abs(price - ref) < 1e-4 * abs(ref) + 2e-7 * float(np.max(p.spot))


@pytest.mark.parametrize("engine", ["cuda", "tc"])
def test_full_heterogeneous_batch_mixed(tp, batch, engine):
    rc, prices, diags = _run(tp, batch, "mixed", engine)
    status = np.array([d.status for d in diags])
    assert np.all((status == tp.TT_OK) | (status == tp.TT_WARN_NOT_CONVERGED))
    assert np.all(np.isfinite(prices)) and np.all(prices > 0)
    imag = np.abs(np.array([d.imag_part for d in diags]))
    ok = status == tp.TT_OK
    assert np.all(imag[ok] <= 1e-2 * prices[ok])
    assert np.all(imag <= 0.5 * prices)
    assert sum(d.terms for d in diags) == sum(p.d if p.payoff == "max" else 1 for p in batch)
    # the stratified sample, priced inside this one launch of 4096
    tier1, tier2 = _golden()
    assert len(tier1) >= 12
    for c in tier1 + tier2:
        i = c["index"]
        assert _mixed_ok(prices[i], c["oracle"], batch[i]), (engine, c["d"], c["n_grid"], c["payoff"], i,
                                                             prices[i], c["oracle"])


def test_stratified_sample_fp64(tp, batch):
    """The first-tier cells in FP64 (one launch of the sample, in the full batch's
    launch configuration): 1e-6 against the oracle."""
    tier1, _ = _golden()
    sub = [batch[c["index"]] for c in tier1]
    rc, prices, diags = _run(tp, sub, "fp64")
    for c, v, dg in zip(tier1, prices, diags):
        assert dg.status in (tp.TT_OK, tp.TT_WARN_NOT_CONVERGED)
        assert math.isfinite(v) and abs(v / c["oracle"] - 1) < 1e-6, (c["d"], c["n_grid"], c["payoff"], v,
                                                                       c["oracle"])
        if "exact_grid" in c:
            assert abs(v / c["exact_grid"] - 1) < 1e-6


@pytest.mark.parametrize("engine", ["cuda", "tc"])
def test_mixed_estimate_guard(tp, batch, engine):
    """The mixed path's estimate checks on the hardest draws (max-calls with d >= 8
    at rank 32, where FP32 half-sweeps can amplify rounding), stopped after 1 to 3
    half-sweeps: a price reported as OK or not converged is a plausible one, in
    (0, sum of spots] with an imaginary part at most 1/4 of it (every train's
    share is checked that way, and the shares are positive); otherwise the
    problem is a numeric error saying that no half-sweep estimate was plausible."""
    idx = [i for i, p in enumerate(batch) if p.payoff == "max" and p.d >= 8 and p.max_rank == 32][:48]
    sub = [batch[i] for i in idx]
    for hs in (1, 2, 3):
        pr = tp.Pricer(max_d=10, max_n=256, max_rank=32, max_batch=len(sub), precision="mixed",
                       engine=engine, max_half_sweeps=hs)
        rc, prices, diags = pr.evaluate(sub)
        pr.close()
        for p, v, dg in zip(sub, prices, diags):
            if dg.status in (tp.TT_OK, tp.TT_WARN_NOT_CONVERGED):
                assert 0 < v <= float(np.sum(p.spot)) and abs(dg.imag_part) <= 0.25 * v, (hs, v, dg)
            else:
                assert dg.status == tp.TT_ERR_NUMERIC and dg.fail_step == 8, (hs, dg)
