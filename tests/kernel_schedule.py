"""Replay of the CUDA kernel's own pivot schedule, for debugging pivot divergence.

Not the oracle.  The oracle (``oracle/ttcross.py``) follows the paper's order:
whole-fiber elimination for the starting rows and whole-fiber maxvol.  The
CUDA kernel reaches rows of the same quality by a cheaper schedule, and in FP64
two different schedules give trains that agree to their TT approximation error,
not to rounding.  When a GPU price parts from the oracle's by more than that,
this module separates pivot choice from arithmetic: it runs the kernel's
schedule in FP64 NumPy on the oracle's integrand, so the FP64 kernel must
reproduce it to rounding (see tests/test_gpu_parity.py).

The kernel's schedule, per core:
  * starting rows from a flat elimination tournament: the current winners
    stacked on top of the next candidates, GEPP keeps the pivot rows.  The
    candidates are the next ``block_rows`` rows for fibers of at most 512 rows;
    larger fibers are screened in blocks of 1024 rows, each 128-row sub-block
    offering its 16 rows with the largest entries (by log-magnitude, ties to the
    lower row);
  * a rank reveal of the winners' pivot block: columns numerically absent from
    the block are dropped, then complete pivoting on the column-equilibrated
    block stops at theta;
  * cyclic block maxvol: B = A_c A_c[W]^{-1} block by block, at most rank-many
    swaps per block visit, until a full cycle has no swap or 4 * n_blocks visits.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from oracle.ttcross import CrossOptions, _fiber, column_scaled, gepp_select


@dataclass
class ScheduleOptions(CrossOptions):
    block_rows: int = 128


SCREEN_MIN_ROWS = 512   # fibers with more rows than this are screened
SCREEN_BLOCK = 1024     # rows per screening block (one GEPP merge each)
SCREEN_SUB = 128        # rows per sub-block
SCREEN_KEEP = 16        # rows each sub-block keeps (a fiber of more than 512 rows offers >= 64)


def screen_rows(a_mat, start, stop):
    """Candidates of one screening block: in every 128-row sub-block, the 16 rows
    whose largest log|entry| (over all columns) is largest, ties to the lower
    row; returned in ascending row order."""
    with np.errstate(divide="ignore"):
        keys = np.log(np.abs(a_mat[start:stop])).max(axis=1)
    kept = []
    for s0 in range(0, stop - start, SCREEN_SUB):
        sub = list(range(s0, min(stop - start, s0 + SCREEN_SUB)))
        best = sorted(sub, key=lambda r: (-float(keys[r]), r))[:SCREEN_KEEP]
        kept += [start + r for r in sorted(best)]
    return kept


def tournament_select(a_mat, block_rows, theta, screen_mat=None):
    """Flat GEPP tournament; returns (winner rows, kept columns).

    Each merge runs GEPP on the current winners stacked on top of new
    candidates: the next block of ``block_rows`` rows when the fiber has at most
    SCREEN_MIN_ROWS rows, else the screened rows of the next SCREEN_BLOCK rows
    (screening keys from ``screen_mat``, default ``a_mat``).
    """
    m = a_mat.shape[0]
    keys_from = a_mat if screen_mat is None else screen_mat
    winners, cols = [], []
    step = block_rows if m <= SCREEN_MIN_ROWS else SCREEN_BLOCK
    for start in range(0, m, step):
        stop = min(m, start + step)
        fresh = list(range(start, stop)) if m <= SCREEN_MIN_ROWS else screen_rows(keys_from, start, stop)
        cand = winners + fresh
        r, c = gepp_select(a_mat[cand, :], theta)
        winners = [cand[p] for p in r]
        cols = c
    return winners, cols


def rank_reveal(p_mat, theta, col_ref=None):
    """Rank-revealing reduction of the pivot block; returns (rows, cols) in pivot order.

    1. A column whose largest |entry|^2 in the block is at most theta^2 times
       ``col_ref`` (its largest |entry|^2 over the whole fiber column) is
       numerically absent from the block and is dropped.
    2. Gaussian elimination with complete pivoting on the column-equilibrated
       block: every entry's |.|^2 is divided by its column's largest in the
       block, at every step the largest such value of the remaining block
       (first in row-major order on ties) is the pivot, and the reduction stops
       when it is at most theta^2.
    Both rules are invariant under column scaling, as the interpolation is; the
    kept sub-block has condition number about 1/theta after column
    equilibration, which the tournament's partial pivoting alone does not
    guarantee."""
    s = np.array(p_mat, dtype=np.complex128, copy=True)
    q, n = s.shape
    blockmax = (s.real ** 2 + s.imag ** 2).max(axis=0)
    keep = blockmax > 0
    if col_ref is not None:
        keep &= blockmax > theta * theta * np.asarray(col_ref, dtype=np.float64)
    scale = np.where(keep, blockmax, np.inf)  # a dropped column never pivots
    free_r = np.ones(q, dtype=bool)
    free_c = np.ones(n, dtype=bool)
    rows, cols = [], []
    while free_r.any() and free_c.any():
        mag = (s.real ** 2 + s.imag ** 2) / scale[None, :]
        mag[~free_r, :] = -1.0
        mag[:, ~free_c] = -1.0
        p, c = divmod(int(np.argmax(mag)), n)
        if not (mag[p, c] > theta * theta):
            break
        rows.append(p)
        cols.append(c)
        free_r[p] = False
        free_c[c] = False
        mult = s[:, c] / s[p, c]
        mult[~free_r] = 0.0
        s -= np.outer(mult, s[p, :])
    return rows, cols


def maxvol_refine(a_cols, rows, block_rows, tau):
    """Cyclic block maxvol on the kept columns, starting from ``rows``.

    Returns (rows, swaps, converged).
    """
    m, rho = a_cols.shape
    rows = list(rows)
    nb = -(-m // block_rows)
    thr = (1.0 + tau) ** 2
    quiet = visits = swaps = 0
    beta = 0
    while quiet < nb and visits < 4 * nb:
        blk = list(range(beta * block_rows, min(m, (beta + 1) * block_rows)))
        inv = np.linalg.inv(a_cols[rows, :])
        b_mat = a_cols[blk, :] @ inv
        swapped = False
        for _ in range(rho):
            mag = b_mat.real ** 2 + b_mat.imag ** 2
            flat = int(np.argmax(mag))
            i, j = divmod(flat, rho)
            if not (mag[i, j] > thr):
                break
            rows[j] = blk[i]
            piv = b_mat[i, j]
            col = b_mat[:, j].copy()
            row = b_mat[i, :].copy()
            row[j] -= 1.0
            b_mat -= np.outer(col, row) / piv
            swapped = True
            swaps += 1
        quiet = 0 if swapped else quiet + 1
        visits += 1
        beta = (beta + 1) % nb
    return rows, swaps, quiet >= nb


def schedule_select(tensor, d, n, k, outer, cols, direction, opts, diag):
    """The kernel's matrix cross step at core k (``select`` for ``oracle.ttcross.tt_cross_sum``);
    returns (new index set, summed interpolant, interpolation core)."""
    raw = _fiber(tensor, d, n, k, outer, cols, direction)
    diag.evaluations += raw.size
    a_mat = column_scaled(raw)
    rows, keep = tournament_select(a_mat, opts.block_rows, opts.theta, screen_mat=raw)
    if not rows:
        raise FloatingPointError("fiber matrix has numerical rank 0")
    col_ref = (a_mat.real ** 2 + a_mat.imag ** 2).max(axis=0)[keep]
    pr, pc = rank_reveal(a_mat[rows][:, keep], opts.theta, col_ref)
    rows, keep = [rows[i] for i in pr], [keep[j] for j in pc]
    a_cols = a_mat[:, keep]
    rows, swaps, ok = maxvol_refine(a_cols, rows, opts.block_rows, opts.tau)
    diag.swaps += swaps
    diag.maxvol_unconverged += 0 if ok else 1
    g = a_cols @ np.linalg.inv(a_cols[rows, :])
    core = g.reshape(len(outer), n, len(rows))
    gsum = core.sum(axis=1)
    if direction == "lr":
        new_set = [tuple(outer[w // n]) + (w % n,) for w in rows]
    else:
        new_set = [(w % n,) + tuple(outer[w // n]) for w in rows]
    return new_set, gsum, core




def replay_price(problem, opts=None):
    """The price by the kernel's schedule: (price, imag, diags)."""
    from oracle.ttcross import tt_price

    return tt_price(problem, opts or ScheduleOptions(), select=schedule_select)
