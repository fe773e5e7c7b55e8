"""Autotuner: candidate sets, the selection rule, the cache round trip (CPU), and
one tuning run on the GPU whose winner prices like the oracle."""
import numpy as np
import pytest

from paper_2203_02804_gb300 import autotune, inputs


def test_candidates_respect_rank_and_precision():
    assert autotune.candidates("fp64", 32) == [{"block_rows": 128, "engine": "cuda"},
                                               {"block_rows": 64, "engine": "cuda"}]
    c = autotune.candidates("mixed", 64)
    assert {(x["block_rows"], x["engine"]) for x in c} == {(128, "cuda"), (128, "tc"), (64, "cuda"), (64, "tc")}
    assert all(x["block_rows"] == 128 for x in autotune.candidates("mixed", 100))


def test_choose_takes_the_fastest_that_agrees():
    ref = np.array([1.0, 2.0, 3.0])
    table = {(128, "cuda"): (3.0, ref), (128, "tc"): (1.0, ref * (1 + 5e-4)),  # fast but disagrees
             (64, "cuda"): (2.0, ref * (1 + 5e-5)), (64, "tc"): (2.5, ref)}
    cands = autotune.candidates("mixed", 32)
    best, recs = autotune.choose(cands, lambda c: table[(c["block_rows"], c["engine"])], 1e-4)
    assert best == {"block_rows": 64, "engine": "cuda"}
    assert [r["agrees"] for r in recs] == [True, False, True, True]


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
    assert {"block_rows": entry["block_rows"], "engine": entry["engine"]} in autotune.candidates("mixed", 16)
    assert len(entry["records"]) == 4 and all(r["seconds"] > 0 for r in entry["records"])
    assert autotune.lookup("mixed", 3, 32, 16, "min") == {"block_rows": entry["block_rows"], "engine": entry["engine"]}
    ps = inputs.tuning_batch(4, 3, 32, 16)
    pr = ttprice.Pricer.tuned(3, 32, 16, 4, precision="mixed")
    _, prices, _ = pr.evaluate(ps)
    pr.close()
    for p, v in zip(ps, prices):
        ref, _, _ = ttcross.tt_price(p)
        assert abs(v - ref) < 1e-4 * abs(ref) + 2e-7 * float(np.max(p.spot))
