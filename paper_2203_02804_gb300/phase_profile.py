"""Where a CTA's time goes: per-phase clock64() totals of the TT-cross kernel.

    python -m paper_2203_02804_gb300.phase_profile [--batch 1216] [--precision mixed] [--engine cuda] [--rank-tol 1e-5]

Builds a profiling variant of the library (-DTTP_PHASE_TIMERS; thread 0 of each
CTA adds the clock span of each phase, barrier waits included) into a temporary
directory, prices one batch of the d=5 call-on-the-minimum workload, and prints
cycles per price and the share of each phase.  The product library is not
touched.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import tempfile
import time

from . import build, inputs, ttprice

PHASES = ["pair table + axis table", "column shifts", "tournament: evaluation + screening",
          "tournament: GEPP", "tournament: winner rows", "maxvol: P^-1 refresh",
          "maxvol: block evaluation", "rank reveal (complete pivoting)", "maxvol: row sums + block product + argmax",
          "maxvol: swaps", "interpolation solve (FP64)", "  (in block evaluation) tensor-core issue", "end-core sums",
          "job set-up (tables, pivots)", "  (in block evaluation) evaluate + split",
          "  (in block evaluation) row sums"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=1216)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--engine", choices=["auto", "cuda", "tc"], default="auto")
    ap.add_argument("--rank-tol", type=float, default=0.0, help="0: the library default")
    args = ap.parse_args()
    import torch

    tmp = tempfile.mkdtemp(prefix="ttprice_phase_")
    lib = os.path.join(tmp, "libttprice_phase.so")
    subprocess.run([build.nvcc_path(), *build.ARCH, "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                    "-DTTP_PHASE_TIMERS", "-I", build.INCLUDE, "-o", lib,
                    os.path.join(build.CSRC, "ttprice.cu")], check=True)
    ttprice._lib = ttprice.load_library(lib)
    L = ttprice._lib
    L.tt_phase_cycles.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int]
    ps = inputs.five_asset_batch(args.batch)
    pr = ttprice.Pricer(max_d=5, max_n=128, max_rank=32, max_batch=args.batch, precision=args.precision,
                        engine=args.engine, rank_tol=args.rank_tol)
    pr.prepare(ps)
    pr.run()
    torch.cuda.synchronize()
    L.tt_phase_cycles(None, 1)
    t0 = time.perf_counter()
    pr.run()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    buf = (ctypes.c_ulonglong * 24)()
    L.tt_phase_cycles(buf, 0)
    pr.close()
    nested = {i for i, name in enumerate(PHASES) if name.startswith("  (in ")}
    tot = sum(v for i, v in enumerate(buf) if i < len(PHASES) and i not in nested)
    print(json.dumps({"workload": "d5-min-call N=128 rank 32", "precision": args.precision,
                      "engine": args.engine, "rank_tol": args.rank_tol or "default",
                      "batch": args.batch, "prices_per_s": args.batch / dt}))
    for i, name in enumerate(PHASES):
        if buf[i]:
            print(f"{name:44s} {buf[i] / args.batch / 1e6:8.3f} Mcycles/price {100 * buf[i] / tot:6.2f}%")
    if buf[20]:
        print(f"maxvol (CUDA-core engine): {buf[20]} swaps, {buf[19] / buf[20] / 1e3:.1f} kcycles of swap loop "
              f"per swap, {(buf[9] - buf[19]) / 1e3 / args.batch:.1f} kcycles per price of visit tails; "
              f"block product loop {buf[21] / args.batch / 1e6:.3f} Mcycles per price")
    if buf[16]:
        print(f"interpolation solves: {buf[16]}, by refinement {buf[16] - buf[17]} "
              f"({buf[18] / buf[16]:.2f} steps each), by elimination {buf[17]}")


if __name__ == "__main__":
    main()
