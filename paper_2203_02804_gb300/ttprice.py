"""Python binding of the C ABI in include/ttprice.h (ctypes; argument marshalling only).

Every pricing step runs in libttprice.so's CUDA kernels.  PyTorch supplies the
device workspace and the CUDA stream.  There is no CPU fallback: if the library
is missing or CUDA is unavailable the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from collections import abc
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from .build import LIB

TT_OK = 0
TT_WARN_NOT_CONVERGED = 1
TT_ERR_INVALID = -1
TT_ERR_NOT_PD = -2
TT_ERR_STRIP = -3
TT_ERR_CAPACITY = -4
TT_ERR_CUDA = -5
TT_ERR_NUMERIC = -6

TT_MIN_CALL = 0
TT_MAX_CALL = 1
TT_FP64 = 0
TT_MIXED = 1
TT_ENGINE_AUTO = 0
TT_ENGINE_CUDA_CORES = 1
TT_ENGINE_TENSOR_CORES = 2
ENGINES = {"auto": TT_ENGINE_AUTO, "cuda": TT_ENGINE_CUDA_CORES, "tc": TT_ENGINE_TENSOR_CORES}
TT_METHOD_SINGLE_TRAIN = 0
TT_METHOD_TWO_TRAINS = 1
METHODS = {"single": TT_METHOD_SINGLE_TRAIN, "two-train": TT_METHOD_TWO_TRAINS}

EXPORTS = ("tt_price_create", "tt_workspace_bytes", "tt_price_evaluate", "tt_price_prepare",
           "tt_price_run", "tt_price_results", "tt_price_transfer_bytes", "tt_price_destroy",
           "tt_status_string", "tt_price_evaluate_static", "tt_price_pivots", "tt_pivot_record_entries",
           # the surrogate's network kernels (include/ttmlp.h)
           "tt_mlp_forward", "tt_mlp_forward_bf16", "tt_mlp_backward", "tt_mlp_mse", "tt_mlp_adam",
           "tt_mlp_to_bf16", "tt_mlp_ensemble", "tt_mlp_gather", "tt_mlp_forward_tc",
           # measured arithmetic peaks (include/ttprobe.h)
           "tt_probe_fma_peak")

# limits of tt_price_evaluate_static (include/ttprice.h)
TT_STATIC_MAX_BATCH = 64
TT_STATIC_MAX_D = 8
TT_STATIC_MAX_N = 256
TT_STATIC_MAX_RANK = 32


class tt_class_tuning(ctypes.Structure):
    _fields_ = [("d_min", ctypes.c_int), ("d_max", ctypes.c_int), ("n_grid", ctypes.c_int),
                ("max_rank", ctypes.c_int), ("payoff", ctypes.c_int), ("block_rows", ctypes.c_int),
                ("rank_tol", ctypes.c_double)]


TT_MAX_CLASSES = 64


class tt_options(ctypes.Structure):
    _fields_ = [("max_d", ctypes.c_int), ("max_n", ctypes.c_int), ("max_rank", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_half_sweeps", ctypes.c_int), ("sweep_tol", ctypes.c_double),
                ("rank_tol", ctypes.c_double), ("maxvol_tol", ctypes.c_double),
                ("block_rows", ctypes.c_int), ("engine", ctypes.c_int), ("graph", ctypes.c_int),
                ("method", ctypes.c_int), ("device", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("classes", ctypes.POINTER(tt_class_tuning)),
                ("n_classes", ctypes.c_int), ("pivot_io", ctypes.c_int)]


class tt_problem(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("spot", ctypes.POINTER(ctypes.c_double)),
                ("cov", ctypes.POINTER(ctypes.c_double)), ("rate", ctypes.c_double),
                ("maturity", ctypes.c_double), ("strike", ctypes.c_double),
                ("payoff", ctypes.c_int), ("damping", ctypes.POINTER(ctypes.c_double)),
                ("n_grid", ctypes.c_int), ("trunc_L", ctypes.c_double),
                ("max_rank", ctypes.c_int), ("seed", ctypes.c_ulonglong), ("max_rank_phi", ctypes.c_int),
                ("warm_sets", ctypes.POINTER(ctypes.c_ushort))]


class tt_diag(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("half_sweeps", ctypes.c_int),
                ("final_rank_max", ctypes.c_int), ("terms", ctypes.c_int),
                ("evaluations", ctypes.c_longlong), ("maxvol_swaps", ctypes.c_longlong),
                ("block_visits", ctypes.c_longlong), ("fail_step", ctypes.c_int),
                ("maxvol_rollbacks", ctypes.c_int), ("imag_part", ctypes.c_double),
                ("flops", ctypes.c_double), ("est_discretization_err", ctypes.c_double)]


_lib = None


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libttprice.so (built by paper_2203_02804_gb300.build); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: run paper_2203_02804_gb300.build.build() first")
    lib = ctypes.CDLL(p)
    lib.tt_price_create.argtypes = [ctypes.POINTER(tt_options), ctypes.POINTER(ctypes.c_void_p)]
    lib.tt_price_create.restype = ctypes.c_int
    lib.tt_workspace_bytes.argtypes = [ctypes.POINTER(tt_options)]
    lib.tt_workspace_bytes.restype = ctypes.c_size_t
    lib.tt_price_evaluate.argtypes = [ctypes.c_void_p, ctypes.POINTER(tt_problem), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(tt_diag)]
    lib.tt_price_evaluate.restype = ctypes.c_int
    lib.tt_price_prepare.argtypes = [ctypes.c_void_p, ctypes.POINTER(tt_problem), ctypes.c_int]
    lib.tt_price_prepare.restype = ctypes.c_int
    lib.tt_price_run.argtypes = [ctypes.c_void_p]
    lib.tt_price_run.restype = ctypes.c_int
    lib.tt_price_results.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(tt_diag)]
    lib.tt_price_results.restype = ctypes.c_int
    lib.tt_price_transfer_bytes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t),
                                            ctypes.POINTER(ctypes.c_size_t)]
    lib.tt_price_transfer_bytes.restype = ctypes.c_int
    lib.tt_price_destroy.argtypes = [ctypes.c_void_p]
    lib.tt_price_destroy.restype = None
    lib.tt_status_string.argtypes = [ctypes.c_int]
    lib.tt_status_string.restype = ctypes.c_char_p
    lib.tt_price_evaluate_static.argtypes = [ctypes.POINTER(tt_problem), ctypes.c_int, ctypes.c_int,
                                             ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(tt_diag)]
    lib.tt_price_evaluate_static.restype = ctypes.c_int
    lib.tt_price_pivots.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_ushort), ctypes.c_size_t]
    lib.tt_price_pivots.restype = ctypes.c_int
    lib.tt_pivot_record_entries.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.tt_pivot_record_entries.restype = ctypes.c_size_t
    if hasattr(lib, "tt_probe_fma_peak"):  # absent from single-source profiling builds
        lib.tt_probe_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        lib.tt_probe_fma_peak.restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def status_string(code: int) -> str:
    return load_library().tt_status_string(int(code)).decode()


def fma_peak(precision: str, reps: int = 5) -> float:
    """Measured FMA throughput of the current CUDA device in TFLOP/s (include/ttprobe.h)."""
    out = ctypes.c_double()
    rc = load_library().tt_probe_fma_peak(1 if precision == "fp32" else 0, int(reps), ctypes.byref(out))
    if rc != 0:
        raise RuntimeError(f"tt_probe_fma_peak failed ({rc})")
    return float(out.value)


@dataclass
class Diag:
    status: int
    half_sweeps: int
    final_rank_max: int
    terms: int
    evaluations: int
    maxvol_swaps: int
    block_visits: int
    fail_step: int
    maxvol_rollbacks: int
    imag_part: float
    flops: float
    est_discretization_err: float


# tt_diag as a NumPy record (same offsets as the C struct)
DIAG_DTYPE = np.dtype({
    "names": [f for f, _ in tt_diag._fields_],
    "formats": [np.int32 if t is ctypes.c_int else np.int64 if t is ctypes.c_longlong else np.float64
                for _, t in tt_diag._fields_],
    "offsets": [getattr(tt_diag, f).offset for f, _ in tt_diag._fields_],
    "itemsize": ctypes.sizeof(tt_diag),
})


class DiagList(abc.Sequence):
    """The per-problem diagnostics of a batch as a sequence of Diag, converted from
    the C array column by column on first access (a caller that ignores them pays
    nothing)."""

    def __init__(self, carray, n: int):
        self._c = carray
        self._n = n
        self._items = None

    def _materialise(self):
        if self._items is None:
            rec = np.frombuffer(self._c, dtype=DIAG_DTYPE, count=self._n)
            cols = [rec[f].tolist() for f in DIAG_DTYPE.names]
            self._items = [Diag(*row) for row in zip(*cols)]
        return self._items

    def __len__(self):
        return self._n

    def __getitem__(self, i):
        return self._materialise()[i]

    def __iter__(self):
        return iter(self._materialise())


# tt_problem as a NumPy record (same offsets as the C struct; checked by the tests)
PROBLEM_DTYPE = np.dtype({
    "names": ["d", "spot", "cov", "rate", "maturity", "strike", "payoff", "damping", "n_grid",
              "trunc_L", "max_rank", "seed", "max_rank_phi", "warm_sets"],
    "formats": [np.int32, np.uint64, np.uint64, np.float64, np.float64, np.float64, np.int32,
                np.uint64, np.int32, np.float64, np.int32, np.uint64, np.int32, np.uint64],
    "offsets": [0, 8, 16, 24, 32, 40, 48, 56, 64, 72, 80, 88, 96, 104],
    "itemsize": 112,
})


class ProblemBatch:
    """Host arrays of a batch in the C layout, kept alive for the duration of the C calls.

    The per-problem vectors are packed into three contiguous FP64 arrays and the
    tt_problem records are filled column-wise with NumPy.
    """

    def __init__(self, problems: Sequence):
        n = len(problems)
        self.count = n
        self.rec = np.zeros(max(1, n), dtype=PROBLEM_DTYPE)
        if n == 0:
            self.arr = self.rec.ctypes.data_as(ctypes.POINTER(tt_problem))
            return
        d = np.fromiter((len(p.spot) for p in problems), dtype=np.int64, count=n)
        self.spot = np.concatenate([p.spot for p in problems], axis=None, dtype=np.float64)
        self.cov = np.concatenate([p.cov for p in problems], axis=None, dtype=np.float64)
        self.damp = np.concatenate([p.damping for p in problems], axis=None, dtype=np.float64)
        if self.cov.size != int(np.sum(d * d)) or self.damp.size != self.spot.size:
            raise ValueError("each problem needs spot[d], cov[d][d] and damping[d]")
        off1 = np.concatenate([[0], np.cumsum(d)[:-1]])
        off2 = np.concatenate([[0], np.cumsum(d * d)[:-1]])
        r = self.rec
        r["d"] = d
        r["spot"] = self.spot.ctypes.data + 8 * off1
        r["cov"] = self.cov.ctypes.data + 8 * off2
        r["damping"] = self.damp.ctypes.data + 8 * off1
        sc = np.array([(p.rate, p.maturity, p.strike, p.trunc_L) for p in problems], dtype=np.float64)
        r["rate"], r["maturity"], r["strike"], r["trunc_L"] = sc[:, 0], sc[:, 1], sc[:, 2], sc[:, 3]
        ints = np.array([(0 if p.payoff == "min" else 1, p.n_grid, p.max_rank) for p in problems], dtype=np.int64)
        r["payoff"] = np.where(ints[:, 0] == 0, TT_MIN_CALL, TT_MAX_CALL)
        r["n_grid"] = ints[:, 1]
        r["max_rank"] = ints[:, 2]
        r["seed"] = [int(p.seed) & ((1 << 64) - 1) for p in problems]
        r["max_rank_phi"] = [int(getattr(p, "max_rank_phi", 0) or 0) for p in problems]
        # warm-start records (uint16), kept alive with the batch
        self.warm = [None if getattr(p, "warm_sets", None) is None
                     else np.ascontiguousarray(p.warm_sets, dtype=np.uint16) for p in problems]
        r["warm_sets"] = [0 if w is None else w.ctypes.data for w in self.warm]
        self.arr = r.ctypes.data_as(ctypes.POINTER(tt_problem))


def class_table(classes):
    """A C array of tt_class_tuning from dicts with keys d_min, d_max, n_grid, max_rank,
    payoff ("min", "max" or None for either), block_rows and rank_tol (missing: 0)."""
    if len(classes) > TT_MAX_CLASSES:
        raise ValueError(f"at most {TT_MAX_CLASSES} classes")
    arr = (tt_class_tuning * max(1, len(classes)))()
    for c, src in zip(arr, classes):
        c.d_min, c.d_max = int(src.get("d_min", 1)), int(src.get("d_max", 255))
        c.n_grid, c.max_rank = int(src.get("n_grid", 0)), int(src.get("max_rank", 0))
        pay = src.get("payoff")
        c.payoff = -1 if pay is None else (TT_MIN_CALL if pay == "min" else TT_MAX_CALL)
        c.block_rows, c.rank_tol = int(src.get("block_rows", 0)), float(src.get("rank_tol", 0.0))
    return arr


class Pricer:
    """Owns one tt_pricer handle on a CUDA device, with a torch-allocated workspace.

    ``method`` = "single" crosses the product integrand (one train per term);
    "two-train" is the paper's bra-ket form (Section IV, Eq. braket): separate
    trains of the payoff transform and the characteristic function, contracted
    site by site (ranks <= 40, D_phi from Problem.max_rank_phi)."""

    def __init__(self, max_d: int, max_n: int, max_rank: int, max_batch: int,
                 precision: str = "fp64", device: int = 0, stream=None, max_half_sweeps: int = 0,
                 sweep_tol: float = 0.0, rank_tol: float = 0.0, maxvol_tol: float = 0.0,
                 block_rows: int = 0, use_torch_workspace: bool = True, engine: str = "auto",
                 graph: bool = True, method: str = "single", classes=None, lib=None, pivot_io: bool = False):
        import torch  # device memory and streams only

        if not torch.cuda.is_available():
            raise RuntimeError("the tensor-train pricer needs a CUDA device; none is available")
        self.lib = lib or load_library()  # another build of the library (profiling, tests) when given
        self.torch = torch
        self.device = device
        self.opts = tt_options()
        o = self.opts
        o.max_d, o.max_n, o.max_rank, o.max_batch = max_d, max_n, max_rank, max_batch
        o.precision = TT_FP64 if precision == "fp64" else TT_MIXED
        o.max_half_sweeps = max_half_sweeps
        o.sweep_tol, o.rank_tol, o.maxvol_tol = sweep_tol, rank_tol, maxvol_tol
        o.block_rows = block_rows
        o.engine = ENGINES[engine]
        o.graph = 1 if graph else 0
        o.method = METHODS[method]
        o.device = device
        # per-class block_rows / rank_tol (the autotuner's table); the library copies it
        self._classes = class_table(classes or [])
        o.classes = self._classes
        o.n_classes = len(classes or [])
        o.pivot_io = 1 if pivot_io else 0
        self.max_d, self.max_rank = max_d, max_rank
        with torch.cuda.device(device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        o.cuda_stream = ctypes.c_void_p(self.stream.cuda_stream)
        self.workspace = None
        if use_torch_workspace:
            nbytes = self.lib.tt_workspace_bytes(ctypes.byref(o))
            if nbytes == 0:
                raise ValueError("invalid pricer options (tt_workspace_bytes returned 0)")
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=f"cuda:{device}")
            ptr = self.workspace.data_ptr()
            o.workspace = ctypes.c_void_p((ptr + 255) // 256 * 256)
            o.workspace_bytes = nbytes
        h = ctypes.c_void_p()
        rc = self.lib.tt_price_create(ctypes.byref(o), ctypes.byref(h))
        if rc != TT_OK:
            raise RuntimeError(f"tt_price_create failed: {status_string(rc)} ({rc})")
        self.handle = h
        self._batch = None

    @classmethod
    def tuned(cls, max_d: int, max_n: int, max_rank: int, max_batch: int, precision: str = "mixed",
              payoff: str = "min", **kw) -> "Pricer":
        """A pricer with the autotuner's configuration for this shape (paper_2203_02804_gb300.autotune),
        or the defaults when the shape has not been tuned."""
        from . import autotune

        cfg = autotune.lookup(precision, max_d, max_n, max_rank, payoff) or {}
        return cls(max_d, max_n, max_rank, max_batch, precision=precision, **{**cfg, **kw})

    def close(self):
        if getattr(self, "handle", None):
            self.lib.tt_price_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- the C calls, one to one ---
    def prepare(self, problems) -> int:
        """Stage a batch: Problem objects, or a ProblemBatch (host structs built once)."""
        self._batch = problems if isinstance(problems, ProblemBatch) else ProblemBatch(problems)
        return self.lib.tt_price_prepare(self.handle, self._batch.arr, self._batch.count)

    def run(self) -> int:
        return self.lib.tt_price_run(self.handle)

    def results(self):
        n = self._batch.count if self._batch else 0
        prices = (ctypes.c_double * max(1, n))()
        diags = (tt_diag * max(1, n))()
        rc = self.lib.tt_price_results(self.handle, prices, diags)
        return rc, np.frombuffer(prices, dtype=np.float64, count=n).copy(), DiagList(diags, n)

    def transfer_bytes(self):
        """(host-to-device bytes of the last prepare, device-to-host bytes of the last results)."""
        h2d, d2h = ctypes.c_size_t(), ctypes.c_size_t()
        self.lib.tt_price_transfer_bytes(self.handle, ctypes.byref(h2d), ctypes.byref(d2h))
        return int(h2d.value), int(d2h.value)

    def pivots(self, i: int) -> np.ndarray:
        """Final right index sets of problem i of the last run (the warm_sets record
        format of include/ttprice.h); needs pivot_io."""
        terms = self.max_d
        cap = int(self.lib.tt_pivot_record_entries(self.max_d, self.max_rank)) * terms
        buf = (ctypes.c_ushort * max(1, cap))()
        n = self.lib.tt_price_pivots(self.handle, int(i), buf, cap)
        if n < 0:
            raise RuntimeError(f"tt_price_pivots failed: {status_string(n)} ({n})")
        return np.frombuffer(buf, dtype=np.uint16, count=n).copy()

    def evaluate(self, problems):
        """Price a batch (Problem objects, or a ProblemBatch of host structs built once);
        returns (worst status, prices ndarray, sequence of Diag)."""
        batch = problems if isinstance(problems, ProblemBatch) else ProblemBatch(problems)
        n = batch.count
        prices = (ctypes.c_double * max(1, n))()
        diags = (tt_diag * max(1, n))()
        rc = self.lib.tt_price_evaluate(self.handle, batch.arr, n, prices, diags)
        return rc, np.frombuffer(prices, dtype=np.float64, count=n).copy(), DiagList(diags, n)
