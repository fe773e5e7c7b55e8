"""The heterogeneous batch at full size: 4096 problems of uneven d, N and rank,
calls on the minimum and on the maximum mixed 50/50, in one launch.

The whole batch runs in the launch configuration the library uses for any batch;
sampled problems are checked against the FP64 oracle one by one (the mixed path
to 1e-4, the FP64 path to 1e-6), and every price is checked for the properties
that hold at any size: a finite positive price, a status that is OK or
not-converged, and an imaginary part of the grid sum that is small next to the
price (the midpoint grid is symmetric, so the exact grid sum is real and the
imaginary part is TT error).  Many draws cap the rank below what the integrand
needs (rank 8 at d = 10); their sweeps end unconverged with a TT error of up to
tens of percent in either precision, so the tight bound on the imaginary part
applies to converged problems and the loose one only rules out a blow-up."""
import math

import numpy as np
import pytest

from oracle import ttcross
from paper_2203_02804_gb300 import inputs

pytestmark = pytest.mark.gpu


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
    # sampled parity: the cheapest rank-32 problems of each payoff whose FP64
    # oracle sweep converges (then the train's own error is small, so FP32 pivot
    # choices that part from FP64 at near-ties stay inside 1e-4; an unconverged,
    # rank-limited train moves by its TT error with any pivot change), priced one
    # by one by the oracle
    for payoff in ("min", "max"):
        idx = sorted((i for i, p in enumerate(batch) if p.payoff == payoff and p.max_rank == 32),
                     key=lambda i: _cost(batch[i]))
        checked = 0
        for i in idx[:12]:
            ref, _, odiags = ttcross.tt_price(batch[i])
            if not all(dg.converged for dg in odiags):
                continue
            # 1e-4 relative, with the FP32 floor: the integrand's terms are of the
            # spot's size, so single-precision arithmetic leaves ~1e-7 x S0 absolute
            # (a price at 7e-4 of the spot sees it as 1.8e-4 relative)
            s0 = float(np.max(batch[i].spot))
            assert abs(prices[i] - ref) < 1e-4 * abs(ref) + 2e-7 * s0, (payoff, i)
            checked += 1
            if checked == 3:
                break
        assert checked == 3, payoff


def test_heterogeneous_subset_fp64(tp, batch):
    idx = sorted(range(len(batch)), key=lambda i: _cost(batch[i]))[:8]
    sub = [batch[i] for i in idx]
    rc, prices, diags = _run(tp, sub, "fp64")
    for p, v, dg in zip(sub, prices, diags):
        assert dg.status in (tp.TT_OK, tp.TT_WARN_NOT_CONVERGED)
        ref, _, _ = ttcross.tt_price(p)
        assert math.isfinite(v) and abs(v / ref - 1) < 1e-6


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
