"""Plain TT-cross with maxvol pivoting, and the TT contraction with the weights.

Test infrastructure only (see the package docstring).

What the paper fixes (Section IV.A-B) and what is read into it
  * The integrand tensor is approximated by a tensor train (matrix product
    state) built from actual tensor entries by TT-cross: sweep back and forth
    over the cores; at each core solve a matrix cross problem M ~ M(:,J)
    M(I,J)^{-1} M(I,:) with the other index sets fixed, choosing the rows I of
    (quasi-)maximal volume by maxvol, starting from random column sets J.
  * The paper leaves the details to its references.  The readings used here,
    and implemented independently by the CUDA library:
      - core k's fiber matrix A has rows (outer multi-index o, grid index i),
        row number o*N + i, and the opposite index set as columns;
      - initial rows: Gaussian elimination with partial pivoting (GEPP) run as a
        flat tournament: the current winners are stacked on top of the next
        candidates and GEPP keeps the pivot rows.  Candidates are the next block
        of ``block_rows`` rows for fibers of at most 512 rows; larger fibers are
        screened in blocks of 1024 rows, each 128-row sub-block offering its 16
        rows with the largest entries.  A column whose best pivot is at most
        ``theta`` times that column's largest entry is skipped (numerically
        dependent); the pivot block of the winners then drops the columns
        whose block entries are at most theta times their largest fiber entry,
        and is reduced by complete pivoting on its column-equilibrated entries
        (stop at theta), which keeps its condition number near 1/theta; the
        kept columns set the rank;
      - maxvol: B = A_c A_c[W]^{-1} on the kept columns, blocks visited
        cyclically; inside a block, while max |B_ij| > 1 + tau swap row i into
        slot j (rank-one update of B, at most rank-many swaps per block); stop
        after every block has been visited once with no swap (then
        |B| <= 1 + tau on the whole matrix) or after 4 * n_blocks visits;
      - the interpolation core is G = A_c A_c[W]^{-1}; its sum over the grid
        index is what the contraction with the quadrature weights needs;
      - half-sweeps alternate left-to-right / right-to-left; each ends with a
        price estimate and the sweep stops when two consecutive estimates agree
        to ``sweep_tol`` (relative), or after ``max_half_sweeps``;
      - ranks r_k = min(r_max, N^k, N^(d-k)); initial right sets draw distinct
        multi-indices with SplitMix64 around the grid centre, with a spread of
        1.5 standard deviations of the integrand's Gaussian factor per axis
        (slot 0 is the centre), or list all N^(d-k) of them in lexicographic
        order when r_k = N^(d-k).
  * Contraction (Section IV.A, MPS inner product): the weights are eta per axis
    (folded into the tensor's scale), so the weighted sum of the train is the
    product of the per-core sums W_k = sum_i G_k[:, i, :].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .splitmix import pivot_key, splitmix64


@dataclass
class CrossOptions:
    block_rows: int = 128
    theta: float = 1e-8           # relative pivot threshold for skipping a column
    tau: float = 0.05             # maxvol tolerance: stop when |B| <= 1 + tau
    max_half_sweeps: int = 8
    sweep_tol: float = 1e-6


@dataclass
class CrossDiag:
    half_sweeps: int = 0
    converged: bool = False
    evaluations: int = 0
    max_rank: int = 0
    swaps: int = 0
    maxvol_unconverged: int = 0
    history: list = field(default_factory=list)
    ranks: list = field(default_factory=list)
    train: list = None  # with keep_train: the cores of the latest left-to-right half-sweep


# ----------------------------------------------------------------------------
# ranks and initial pivots
# ----------------------------------------------------------------------------

def bond_ranks(d, n, r_max):
    """r_0 = r_d = 1, r_k = min(r_max, N^k, N^(d-k))."""
    return [1] + [min(r_max, n ** k, n ** (d - k)) for k in range(1, d)] + [1]


PEAK_ATTEMPTS = 64
TWO_M53 = 1.0 / 9007199254740992.0  # 2^-53
SQRT3 = math.sqrt(3.0)


def pivot_widths(cov_diag, maturity, eta):
    """Spread of the initial pivots per axis, in grid steps: 1.5 standard
    deviations of the Gaussian factor exp(-T/2 Cov_jj u^2), w_j = 1.5/(sqrt(Cov_jj T) eta)."""
    return [1.5 / (math.sqrt(c * maturity) * eta) for c in cov_diag]


def _peak_coordinate(seed, term, k, t, b, j, n, w):
    """N/2 + round(w z), z ~ (sum of four SplitMix64 uniforms - 2) sqrt(3), clamped."""
    s = 0.0
    for q in range(4):
        s += (splitmix64(pivot_key(seed, term, k, t, b, 4 * j + q)) >> 11) * TWO_M53
    z = (s - 2.0) * SQRT3
    idx = n // 2 + math.floor(w * z + 0.5)
    return min(max(idx, 0), n - 1)


def initial_right_set(d, n, k, size, seed, term, widths=None):
    """Distinct right multi-indices over axes k..d-1 (0-based), ``size`` of them.

    Slot 0 is the grid centre.  The others are random (the paper starts
    TT-cross from random column sets): the first 64 attempts of a slot draw each
    coordinate around the centre with spread ``widths[j]`` (where the
    integrand's Gaussian factor lives); later attempts draw uniformly on the
    grid.  A draw equal to an earlier slot is rejected.  When r_k = N^(d-k)
    the set is every multi-index in lexicographic order.
    """
    width = d - k
    if n ** width == size:
        out = []
        for flat in range(size):
            idx = []
            rem = flat
            for _ in range(width):
                idx.append(rem % n)
                rem //= n
            out.append(tuple(reversed(idx)))
        return out
    out = [tuple([n // 2] * width)]
    seen = {out[0]}
    for b in range(1, size):
        for t in range(65536):
            if widths is not None and t < PEAK_ATTEMPTS:
                cand = tuple(_peak_coordinate(seed, term, k, t, b, j, n, widths[j]) for j in range(k, d))
            else:
                cand = tuple(splitmix64(pivot_key(seed, term, k, t, b, j)) % n for j in range(k, d))
            if cand not in seen:
                break
        else:
            raise RuntimeError("initial pivot draw did not find a fresh multi-index")
        seen.add(cand)
        out.append(cand)
    return out


# ----------------------------------------------------------------------------
# row selection: GEPP tournament and maxvol
# ----------------------------------------------------------------------------

def gepp_select(c_mat, theta):
    """GEPP with partial pivoting on the candidate matrix; returns (rows, cols).

    Columns are taken in order.  The pivot of column c is the available row with
    the largest |entry| of the current Schur complement (first one on ties).  If
    |pivot| <= theta * max_i |original entry of column c|, the column is skipped.
    """
    s = np.array(c_mat, dtype=np.complex128, copy=True)
    q, n = s.shape
    if q == 0:
        return [], []
    colmax = (s.real ** 2 + s.imag ** 2).max(axis=0)
    avail = np.ones(q, dtype=bool)
    rows, cols = [], []
    for c in range(n):
        if not avail.any():
            break
        mag = s[:, c].real ** 2 + s[:, c].imag ** 2
        mag = np.where(avail, mag, -1.0)
        p = int(np.argmax(mag))
        if not (mag[p] > theta * theta * colmax[c]) or mag[p] == 0.0:
            continue
        rows.append(p)
        cols.append(c)
        avail[p] = False
        if c + 1 < n:
            mult = s[:, c] / s[p, c]
            mult[~avail] = 0.0
            s[:, c + 1:] -= np.outer(mult, s[p, c + 1:])
    return rows, cols


SCREEN_MIN_ROWS = 512   # fibers with more rows than this are screened
SCREEN_BLOCK = 1024     # rows per screening block (one GEPP merge each)
SCREEN_SUB = 128        # rows per sub-block
SCREEN_KEEP = 16        # rows each sub-block keeps (a fiber of more than 512 rows offers >= 64)


def screen_rows(a_mat, start, stop):
    """Candidates of one screening block: in every 128-row sub-block, the 16 rows
    whose largest |entry|^2 (over all columns, rounded to FP32) is largest, ties
    to the lower row; returned in ascending row order."""
    keys = (a_mat[start:stop].real ** 2 + a_mat[start:stop].imag ** 2).max(axis=1).astype(np.float32)
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


# ----------------------------------------------------------------------------
# one core of a half-sweep
# ----------------------------------------------------------------------------

def _fiber(tensor, d, n, k, outer, cols, direction):
    """Fiber matrix of core k: rows (o, i) -> o*N + i, columns = ``cols``.

    direction 'lr': full index = outer[o] + (i,) + cols[c]
    direction 'rl': full index = cols[c] + (i,) + outer[o]
    """
    no, nc = len(outer), len(cols)
    idx = np.empty((no, n, nc, d), dtype=np.int64)
    outer_a = np.array(outer, dtype=np.int64).reshape(no, -1)
    cols_a = np.array(cols, dtype=np.int64).reshape(nc, -1)
    grid_i = np.arange(n, dtype=np.int64)
    if direction == "lr":
        idx[..., :k] = outer_a[:, None, None, :]
        idx[..., k] = grid_i[None, :, None]
        idx[..., k + 1:] = cols_a[None, None, :, :]
    else:
        idx[..., :k] = cols_a[None, None, :, :]
        idx[..., k] = grid_i[None, :, None]
        idx[..., k + 1:] = outer_a[:, None, None, :]
    return tensor(idx).reshape(no * n, nc)


def column_scaled(a_mat):
    """Each column times a power of two that brings its largest |entry| into
    (1/2, 1]; all-zero columns unchanged.  Pivot choices, maxvol's B and the
    interpolation core are invariant under column scaling; the scaling keeps
    |a|^2 and the pivot-block inverse inside the FP64 range for fibers through
    far tails.  No pivot decision depends on it: GEPP, maxvol and
    ``rank_reveal`` are invariant under column scaling."""
    cm = np.abs(a_mat).max(axis=0)
    expo = np.where(cm > 0, np.ceil(np.log2(np.where(cm > 0, cm, 1.0))), 0.0)
    return a_mat * np.exp2(-expo)


def core_select(tensor, d, n, k, outer, cols, direction, opts, diag):
    """Select rows of core k's fiber; returns (new index set, summed interpolant,
    interpolation core G = A_c A_c[W]^{-1} as an (outer, N, rank) array)."""
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


def core_sum(tensor, d, n, k, outer, direction, diag, end_core=None):
    """End core of a half-sweep: sum over its grid index, one value per outer index
    (the fiber itself, (outer, N, 1), is appended to ``end_core`` when given)."""
    a_mat = _fiber(tensor, d, n, k, outer, [()], direction)
    diag.evaluations += a_mat.size
    if end_core is not None:
        end_core.append(a_mat.reshape(len(outer), n, 1))
    return a_mat.reshape(len(outer), n).sum(axis=1)


# ----------------------------------------------------------------------------
# the sweeps
# ----------------------------------------------------------------------------

def tt_cross_sum(tensor, r_max, seed, term=0, opts=None, keep_train=False):
    """TT-cross approximation of sum over the grid of ``tensor``; returns (sum, diag).

    With ``keep_train`` the cores of the latest left-to-right half-sweep are kept
    in ``diag.train``: G_0, ..., G_{d-2} (interpolation cores, (r_{k-1}, N, r_k))
    and the end core's fiber (r_{d-2}, N, 1); their product is the train whose
    weighted sum that half-sweep estimated."""
    opts = opts or CrossOptions()
    d, n = tensor.d, tensor.n
    ranks = bond_ranks(d, n, r_max)
    lsets = [None] * (d + 1)
    rsets = [None] * (d + 1)
    lsets[0] = [()]
    rsets[d] = [()]
    widths = getattr(tensor, "pivot_widths", None)
    for k in range(1, d):
        rsets[k] = initial_right_set(d, n, k, ranks[k], seed, term, widths)
    diag = CrossDiag()
    prev = None
    est = 0j
    for s in range(opts.max_half_sweeps):
        if s % 2 == 0:
            v = np.ones(1, dtype=np.complex128)
            cores = []
            for k in range(d - 1):
                lsets[k + 1], gsum, core = core_select(tensor, d, n, k, lsets[k], rsets[k + 1], "lr", opts, diag)
                cores.append(core)
                v = v @ gsum
            est = complex(v @ core_sum(tensor, d, n, d - 1, lsets[d - 1], "lr", diag, cores))
            if keep_train:
                diag.train = cores
        else:
            v = np.ones(1, dtype=np.complex128)
            for k in range(d - 1, 0, -1):
                rsets[k], gsum, _ = core_select(tensor, d, n, k, rsets[k + 1], lsets[k], "rl", opts, diag)
                v = gsum.T @ v
            est = complex(core_sum(tensor, d, n, 0, rsets[1], "rl", diag) @ v)
        diag.half_sweeps = s + 1
        diag.history.append(est)
        sets = lsets[1:d] if s % 2 == 0 else rsets[1:d]
        diag.ranks = [len(x) for x in sets]
        diag.max_rank = max([diag.max_rank, 1] + diag.ranks)
        if d == 1:
            diag.converged = True
            break
        if prev is not None and abs(est - prev) <= opts.sweep_tol * abs(est):
            diag.converged = True
            break
        prev = est
    return est, diag


def tt_price(problem, opts=None):
    """Price = Re(sum over terms of scale * TT-cross sum); returns (price, imag, diags)."""
    from .integrand import tensors_for

    acc = 0j
    diags = []
    for term, t in enumerate(tensors_for(problem)):
        est, dg = tt_cross_sum(t, int(problem.max_rank), int(problem.seed), term, opts)
        acc += t.scale * est
        diags.append(dg)
    return acc.real, acc.imag, diags


def dense_from_cores(cores):
    """Brute-force TT -> dense tensor (for pinning the contraction on tiny cases)."""
    out = cores[0]
    for c in cores[1:]:
        out = np.tensordot(out, c, axes=([-1], [0]))
    return out.reshape(out.shape[1:-1])
