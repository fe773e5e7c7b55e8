"""The C ABI on the CPU: the library builds for sm_103a, loads, exports every
function include/*.h declare, and the ctypes mirrors
of its structs have the C layout (checked against gcc).  No compute call runs
here."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2203_02804_gb300 import build, ttprice

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ttprice.h")
HEADERS = [HEADER, os.path.join(ROOT, "include", "ttmlp.h"), os.path.join(ROOT, "include", "ttprobe.h")]


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ttprice.load_library()


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(tt_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    assert set(names) == set(ttprice.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_without_gpu(lib):
    assert lib.tt_status_string(0) == b"ok"
    assert b"positive definite" in lib.tt_status_string(-2)


def test_create_rejects_bad_options_without_touching_the_gpu(lib):
    o = ttprice.tt_options()
    o.max_d, o.max_n, o.max_rank, o.max_batch = 0, 64, 8, 1  # max_d < 1
    h = ctypes.c_void_p()
    assert lib.tt_price_create(ctypes.byref(o), ctypes.byref(h)) == ttprice.TT_ERR_INVALID
    assert not h.value
    o.max_d, o.max_rank, o.block_rows = 4, 64, 250  # block_rows + max_rank > 256
    assert lib.tt_price_create(ctypes.byref(o), ctypes.byref(h)) == ttprice.TT_ERR_INVALID
    # the tensor-core block product is one 128-row tile; FP64 has no tensor-core engine
    o.max_rank, o.block_rows, o.precision = 32, 160, ttprice.TT_MIXED
    o.engine = ttprice.TT_ENGINE_TENSOR_CORES
    assert lib.tt_price_create(ctypes.byref(o), ctypes.byref(h)) == ttprice.TT_ERR_INVALID
    o.block_rows, o.precision = 128, ttprice.TT_FP64
    assert lib.tt_price_create(ctypes.byref(o), ctypes.byref(h)) == ttprice.TT_ERR_INVALID
    o.engine = 3
    assert lib.tt_price_create(ctypes.byref(o), ctypes.byref(h)) == ttprice.TT_ERR_INVALID
    # the two-train form: a method out of range, or ranks above its 32
    o.engine, o.method = ttprice.TT_ENGINE_AUTO, 2
    assert lib.tt_price_create(ctypes.byref(o), ctypes.byref(h)) == ttprice.TT_ERR_INVALID
    o.method, o.max_rank, o.block_rows = ttprice.TT_METHOD_TWO_TRAINS, 64, 128
    assert lib.tt_price_create(ctypes.byref(o), ctypes.byref(h)) == ttprice.TT_ERR_INVALID
    # the per-class table: too many classes, a missing table, a class block taller than the options'
    o.method, o.max_rank, o.block_rows, o.engine = ttprice.TT_METHOD_SINGLE_TRAIN, 16, 64, ttprice.TT_ENGINE_AUTO
    o.max_d = 4
    tbl = ttprice.class_table([{"max_rank": 16, "block_rows": 128}])
    o.classes, o.n_classes = tbl, 1
    assert lib.tt_price_create(ctypes.byref(o), ctypes.byref(h)) == ttprice.TT_ERR_INVALID
    o.n_classes = ttprice.TT_MAX_CLASSES + 1
    assert lib.tt_price_create(ctypes.byref(o), ctypes.byref(h)) == ttprice.TT_ERR_INVALID
    o.classes, o.n_classes = None, 1
    assert lib.tt_price_create(ctypes.byref(o), ctypes.byref(h)) == ttprice.TT_ERR_INVALID
    assert not h.value
    lib.tt_price_destroy(None)


def test_class_table_marshalling():
    t = ttprice.class_table([{"d_min": 3, "d_max": 6, "n_grid": 128, "max_rank": 32, "payoff": "max",
                              "block_rows": 64, "rank_tol": 3e-6}, {"max_rank": 8}])
    assert (t[0].d_min, t[0].d_max, t[0].n_grid, t[0].max_rank) == (3, 6, 128, 32)
    assert t[0].payoff == ttprice.TT_MAX_CALL and t[0].block_rows == 64 and t[0].rank_tol == 3e-6
    assert t[1].payoff == -1 and (t[1].d_min, t[1].d_max) == (1, 255) and t[1].block_rows == 0


def test_struct_layouts_match_c():
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "ttprice.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(tt_options), offsetof(tt_options, sweep_tol),
             offsetof(tt_options, block_rows), offsetof(tt_options, engine), offsetof(tt_options, graph),
             offsetof(tt_options, method), offsetof(tt_options, cuda_stream),
             offsetof(tt_options, workspace_bytes));
      printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(tt_problem), offsetof(tt_problem, rate),
             offsetof(tt_problem, damping), offsetof(tt_problem, trunc_L), offsetof(tt_problem, seed),
             offsetof(tt_problem, max_rank_phi), offsetof(tt_problem, warm_sets));
      printf("%zu %zu %zu %zu %zu\n", sizeof(tt_diag), offsetof(tt_diag, evaluations), offsetof(tt_diag, fail_step),
             offsetof(tt_diag, flops), offsetof(tt_diag, est_discretization_err));
      printf("%zu %zu %zu %zu\n", sizeof(tt_class_tuning), offsetof(tt_class_tuning, rank_tol),
             offsetof(tt_options, n_classes), offsetof(tt_options, pivot_io));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as tmp:
        c = os.path.join(tmp, "layout.c")
        exe = os.path.join(tmp, "layout")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    T = ttprice
    want = [
        [ctypes.sizeof(T.tt_options), T.tt_options.sweep_tol.offset, T.tt_options.block_rows.offset,
         T.tt_options.engine.offset, T.tt_options.graph.offset, T.tt_options.method.offset,
         T.tt_options.cuda_stream.offset, T.tt_options.workspace_bytes.offset],
        [ctypes.sizeof(T.tt_problem), T.tt_problem.rate.offset, T.tt_problem.damping.offset,
         T.tt_problem.trunc_L.offset, T.tt_problem.seed.offset, T.tt_problem.max_rank_phi.offset,
         T.tt_problem.warm_sets.offset],
        [ctypes.sizeof(T.tt_diag), T.tt_diag.evaluations.offset, T.tt_diag.fail_step.offset,
         T.tt_diag.flops.offset, T.tt_diag.est_discretization_err.offset],
        [ctypes.sizeof(T.tt_class_tuning), T.tt_class_tuning.rank_tol.offset, T.tt_options.n_classes.offset,
         T.tt_options.pivot_io.offset],
    ]
    assert len([ln for ln in out if ln.strip()]) == len(want)
    for line, w in zip(out, want):
        assert [int(v) for v in line.split()] == w


def test_numpy_problem_record_matches_ctypes():
    T = ttprice
    assert T.PROBLEM_DTYPE.itemsize == ctypes.sizeof(T.tt_problem)
    for name, _ in T.tt_problem._fields_:
        assert T.PROBLEM_DTYPE.fields[name][1] == getattr(T.tt_problem, name).offset, name


def test_problem_batch_packs_pointers():
    import numpy as np

    from paper_2203_02804_gb300 import inputs

    ps = [inputs.two_asset_min_call(), inputs.five_asset_batch(1)[0], inputs.two_asset_min_call(payoff="max")]
    b = ttprice.ProblemBatch(ps)
    for i, p in enumerate(ps):
        rec = b.arr[i]
        assert rec.d == p.d and rec.n_grid == p.n_grid and rec.max_rank == p.max_rank
        assert [rec.spot[j] for j in range(p.d)] == list(np.asarray(p.spot, dtype=float))
        assert [rec.cov[j] for j in range(p.d * p.d)] == list(np.asarray(p.cov, dtype=float).ravel())
        assert [rec.damping[j] for j in range(p.d)] == list(np.asarray(p.damping, dtype=float))
        assert rec.payoff == (ttprice.TT_MIN_CALL if p.payoff == "min" else ttprice.TT_MAX_CALL)
        assert rec.seed == p.seed


def test_problem_batch_packs_every_field():
    """The packed tt_problem records point at each problem's own spot, covariance
    and damping values and carry its scalars (heterogeneous d, both payoffs)."""
    from paper_2203_02804_gb300 import inputs

    probs = inputs.mixed_batch(24)
    b = ttprice.ProblemBatch(probs)
    assert b.count == len(probs)
    dbl = ctypes.POINTER(ctypes.c_double)
    for p, r in zip(probs, b.rec):
        d = p.d
        assert int(r["d"]) == d
        for name, want in (("spot", p.spot), ("cov", np.ravel(p.cov)), ("damping", p.damping)):
            got = np.ctypeslib.as_array(ctypes.cast(int(r[name]), dbl), shape=(np.size(want),))
            assert np.array_equal(got, np.asarray(want, dtype=np.float64)), name
        assert float(r["rate"]) == p.rate and float(r["maturity"]) == p.maturity
        assert float(r["strike"]) == p.strike and float(r["trunc_L"]) == p.trunc_L
        assert int(r["payoff"]) == (ttprice.TT_MIN_CALL if p.payoff == "min" else ttprice.TT_MAX_CALL)
        assert int(r["n_grid"]) == p.n_grid and int(r["max_rank"]) == p.max_rank
        assert int(r["seed"]) == p.seed and int(r["max_rank_phi"]) == p.max_rank_phi
        assert int(r["warm_sets"]) == 0


def test_diag_list_reads_the_c_array():
    """Per-problem diagnostics come back as a sequence of Diag read from the C
    array (all field types: int, long long, double)."""
    c = (ttprice.tt_diag * 3)()
    c[1].status, c[1].evaluations, c[1].fail_step = ttprice.TT_ERR_NUMERIC, 123456789012, 9
    c[2].imag_part, c[2].maxvol_rollbacks, c[2].flops, c[2].terms = -0.25, 7, 1.5e12, 10
    dl = ttprice.DiagList(c, 3)
    assert len(dl) == 3
    assert dl[1].status == ttprice.TT_ERR_NUMERIC and dl[1].evaluations == 123456789012 and dl[1].fail_step == 9
    assert dl[2].imag_part == -0.25 and dl[2].maxvol_rollbacks == 7 and dl[2].flops == 1.5e12
    assert [d.terms for d in dl] == [0, 0, 10]
    assert dl[-1] == dl[2] and len(dl[:2]) == 2
