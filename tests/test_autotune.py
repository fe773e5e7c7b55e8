"""Autotuner: candidate sets, the selection rule, the cache round trip (CPU), and
one tuning run on the GPU whose winner prices like the oracle."""
import numpy as np
import pytest

from paper_2203_02804_gb300 import autotune, inputs


def test_candidates_respect_rank_and_precision():
    assert autotune.candidates("fp64", 32) == [{"block_rows": 128, "engine": "cuda", "rank_tol": 1e-8},
                                               {"block_rows": 64, "engine": "cuda", "rank_tol": 1e-8}]
    c = autotune.candidates("mixed", 32)
    assert len(c) == 12  # block rows x engine x rank threshold
    assert {(x["block_rows"], x["engine"]) for x in c} == {(128, "cuda"), (128, "tc"), (64, "cuda"), (64, "tc")}
    assert {x["rank_tol"] for x in c} == {1e-6, 3e-6, 1e-5}
    assert all(x["block_rows"] == 128 for x in autotune.candidates("mixed", 100))
    assert {x["engine"] for x in autotune.candidates("mixed", 16, engines=("cuda",))} == {"cuda"}


def test_choose_takes_the_fastest_the_fp64_reference_accepts():
    ref = np.array([1.0, 2.0, 3.0])
    spot = np.array([100.0, 100.0, 100.0])
    cands = autotune.candidates("mixed", 32)
    # the loosest threshold is fastest but 5e-4 off; 64-row tensor cores at 3e-6 is next
    def measure(c):
        secs = {1e-6: 3.0, 3e-6: 2.0, 1e-5: 1.0}[c["rank_tol"]] + (0.1 if c["block_rows"] == 128 else 0.0) \
            + (0.05 if c["engine"] == "cuda" else 0.0)
        err = 5e-4 if c["rank_tol"] == 1e-5 else 5e-5
        return secs, ref * (1 + err)
    best, recs = autotune.choose(cands, measure, ref, spot, "mixed")
    assert best == {"block_rows": 64, "engine": "tc", "rank_tol": 3e-6}
    assert sum(r["agrees"] for r in recs) == 8
    # the FP32 floor: a tiny price may be off by 2e-7 of the spot
    assert autotune.accepted(np.array([1e-3 + 1e-5]), np.array([1e-3]), np.array([100.0]), "mixed")
    assert not autotune.accepted(np.array([1e-3 + 1e-4]), np.array([1e-3]), np.array([100.0]), "mixed")
    # within the tolerance but past its margin (the served batch is not the sample): refused
    assert not autotune.accepted(ref * (1 + 8e-5), ref, spot, "mixed")
    assert autotune.error_ratio(ref * (1 + 8e-5), ref, spot, "mixed") < 1.0
    # nothing accepted: the tightest threshold, fastest of those
    best, _ = autotune.choose(cands, lambda c: (1.0 if c["block_rows"] == 64 else 2.0, ref * 1.1), ref, spot, "mixed")
    assert best["rank_tol"] == 1e-6 and best["block_rows"] == 64


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "t.json")
    k = autotune.shape_key("103", "mixed", 5, 128, 32, "min")
    assert k == "sm_103|mixed|d5|N128|r32|min"
    autotune.store(k, {"block_rows": 64, "engine": "tc", "records": []}, p)
    autotune.store("other", {"block_rows": 128, "engine": "cuda"}, p)
    c = autotune.load_cache(p)
    assert c[k]["engine"] == "tc" and c["other"]["block_rows"] == 128


def test_tuning_batch_is_seeded_and_shaped():
    a = inputs.tuning_batch(3, 4, 32, 8, "max")
    b = inputs.tuning_batch(3, 4, 32, 8, "max")
    assert all(np.array_equal(x.spot, y.spot) for x, y in zip(a, b))
    assert all(x.d == 4 and x.n_grid == 32 and x.max_rank == 8 and x.payoff == "max" for x in a)
    assert inputs.tuning_batch(1, 20, 64, 8)[0].damping[0] == pytest.approx(-0.25)


@pytest.mark.gpu
def test_gpu_tuning_run_and_tuned_pricer(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import ttcross
    from paper_2203_02804_gb300 import build, ttprice

    build.build()
    monkeypatch.setenv("TTPRICE_TUNING_CACHE", str(tmp_path / "tune.json"))
    entry = autotune.tune("mixed", 3, 32, 16, "min")
    assert {k: entry[k] for k in autotune.KNOBS} in autotune.candidates("mixed", 16)
    assert len(entry["records"]) == 12 and all(r["seconds"] > 0 for r in entry["records"])
    assert autotune.lookup("mixed", 3, 32, 16, "min") == {k: entry[k] for k in autotune.KNOBS}
    ps = inputs.tuning_batch(4, 3, 32, 16)
    pr = ttprice.Pricer.tuned(3, 32, 16, 4, precision="mixed")
    _, prices, _ = pr.evaluate(ps)
    pr.close()
    for p, v in zip(ps, prices):
        ref, _, _ = ttcross.tt_price(p)
        assert abs(v - ref) < 1e-4 * abs(ref) + 2e-7 * float(np.max(p.spot))


@pytest.mark.gpu
def test_gpu_class_tuning_drives_one_heterogeneous_launch():
    """Per-class tuning of a small heterogeneous batch: a table entry per (rank cap,
    payoff) class, and one launch with that table prices the batch like the FP64
    path (to 1e-4 on most problems; rank-limited trains differ by their TT error)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_02804_gb300 import build, ttprice

    build.build()
    batch = [p for p in inputs.mixed_batch(400) if p.d <= 6 and p.n_grid <= 128][:96]
    table, recs = autotune.tune_classes("mixed", batch, sample=48, reps=1)
    assert len(table) == len({(p.max_rank, p.payoff) for p in batch})
    for t in table:
        assert t["block_rows"] >= t["max_rank"] and t["rank_tol"] in autotune.RANK_TOLS["mixed"]
    kw = dict(max_d=6, max_n=128, max_rank=32, max_batch=len(batch))
    pr = ttprice.Pricer(precision="fp64", **kw)
    _, ref, _ = pr.evaluate(batch)
    pr.close()
    pr = ttprice.Pricer(precision="mixed", engine="cuda", classes=table, **kw)
    _, got, diags = pr.evaluate(batch)
    pr.close()
    ok = np.array([d.status in (ttprice.TT_OK, ttprice.TT_WARN_NOT_CONVERGED) for d in diags])
    assert ok.all()
    # rank-limited trains part from the FP64 path by their TT error; most are converged
    rel = np.abs(got / ref - 1)
    assert np.median(rel) < 1e-4 and np.all(rel < 5e-2)


def test_error_ratio_edge_cases():
    ref = np.array([1.0, 2.0])
    spot = np.array([100.0, 100.0])
    # a non-finite price refuses the candidate whatever the others do
    assert autotune.error_ratio(np.array([1.0, np.nan]), ref, spot, "mixed") == float("inf")
    assert not autotune.accepted(np.array([1.0, np.inf]), ref, spot, "mixed")
    # only the problems of the mask count (unconverged FP64 references say nothing)
    off = np.array([1.0 + 1e-2, 2.0])
    assert autotune.error_ratio(off, ref, spot, "mixed", mask=np.array([False, True])) == 0.0
    assert autotune.error_ratio(off, ref, spot, "mixed", mask=np.array([False, False])) == 0.0
    # in units of the tolerance: 1e-4 relative + 2e-7 x spot
    r = autotune.error_ratio(np.array([1.0 + 6e-5]), np.array([1.0]), np.array([100.0]), "mixed")
    assert abs(r - 6e-5 / (1e-4 + 2e-5)) < 1e-9
    assert autotune.error_ratio(np.array([]), np.array([]), np.array([]), "mixed") == 0.0
