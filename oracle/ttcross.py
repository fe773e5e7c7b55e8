"""Plain TT-cross with maxvol pivoting, and the TT contraction with the weights.

Test infrastructure only (see the package docstring).

The algorithm, in the paper's order (Section IV.B)
  * The integrand tensor is approximated by a tensor train (matrix product
    state) built from actual tensor entries.  Sweeping back and forth over the
    cores with the other index sets fixed, each core solves one matrix cross
    problem M ~ M(:,J) M(I,J)^{-1} M(I,:): starting from the column set J (at
    first random), it takes the r rows of (quasi-)maximal volume in M(:,J) by
    maxvol; those rows are the next core's row index set, and the sweep in the
    other direction does the same for the columns.
  * maxvol (Goreinov-Tyrtyshnikov, the paper's maxvol reference): start from r
    rows with a non-singular r x r block (Gaussian elimination with partial
    pivoting, the usual start), form B = A A[I]^{-1} over all rows of the fiber,
    and while some |B_ij| > 1 + tau swap row i into slot j (a rank-one update
    of B; every swap multiplies |det A[I]| by |B_ij|).  It stops with
    |B| <= 1 + tau on the whole fiber.  As in the TT-cross references the paper
    cites, maxvol runs on an orthonormal basis of the fiber's columns (QR):
    B, and hence the rows, are the same for any basis of the same column span.
  * Convergence: the paper checks a sampled one-norm after each sweep; here
    each half-sweep ends with the estimate of the weighted sum it computes,
    and the sweeps stop when two consecutive estimates agree to ``sweep_tol``
    (relative) or after ``max_half_sweeps``.
  * Contraction (Section IV.A, MPS inner product): the weights are eta per axis
    (folded into the tensor's scale), so the weighted sum of the train is the
    product of the per-core sums W_k = sum_i G_k[:, i, :] of the interpolation
    cores G_k = A_k A_k[I_k]^{-1}.

Readings where the paper leaves details to its references
  * Core k's fiber matrix has rows (outer multi-index o, grid index i), row
    number o*N + i, and the opposite index set as columns.
  * Rank: the paper fixes the bond dimension D.  Where the fiber matrix has
    numerical rank below its column count, A[I] would be singular.  The QR is
    therefore column-pivoted (rank revealing): the rank r_k is the count of
    |R_kk| > theta |R_00| and the first r_k pivot columns are kept.  Ranks start
    at r_k = min(D, N^k, N^(d-k)) and can only fall.
  * Column scaling: every fiber column is scaled by a power of two that brings
    its largest entry near one, before the QR.  It equilibrates the columns
    for the rank decision (the column-pivoted QR compares column norms) and
    keeps |a|^2 inside the FP64 range for fibers through far tails; maxvol's B
    and the interpolation core are invariant under it.
  * Initial column sets: distinct multi-indices drawn with SplitMix64 around
    the grid centre, with a spread of 1.5 standard deviations of the
    integrand's Gaussian factor per axis (slot 0 is the centre), or all
    N^(d-k) of them in lexicographic order when r_k = N^(d-k).
  * maxvol's tolerance tau (0.05) and a swap cap of 100 r per core (never
    reached in the tests; reaching it is reported in the diagnostics).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from .splitmix import pivot_key, splitmix64


@dataclass
class CrossOptions:
    theta: float = 1e-8           # relative pivot threshold for skipping a column
    tau: float = 0.05             # maxvol tolerance: stop when |B| <= 1 + tau
    max_half_sweeps: int = 8
    sweep_tol: float = 1e-6
    swap_cap: int = 100           # maxvol swaps per core at most swap_cap * rank


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
# row selection: elimination start and maxvol
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


def maxvol(a_cols, rows, tau, max_swaps):
    """maxvol on the whole tall matrix ``a_cols`` (m x r), starting from ``rows``.

    B = A A[rows]^{-1}; while max |B_ij| > 1 + tau: row i replaces slot j and B
    takes the rank-one update B -= B[:, j] (B[i, :] - e_j) / B[i, j].  Returns
    (rows, swaps, converged); converged means |B| <= 1 + tau everywhere.
    """
    rows = list(rows)
    b_mat = a_cols @ np.linalg.inv(a_cols[rows, :])
    r = len(rows)
    for swaps in range(max_swaps + 1):
        mag = np.abs(b_mat)
        i, j = divmod(int(np.argmax(mag)), r)
        if not (mag[i, j] > 1.0 + tau):
            return rows, swaps, True
        if swaps == max_swaps:
            break
        rows[j] = i
        row = b_mat[i, :].copy()
        row[j] -= 1.0
        b_mat -= np.outer(b_mat[:, j], row) / b_mat[i, j]
    return rows, max_swaps, False


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
    """One matrix cross step at core k: fiber, its column basis, maxvol, interpolation core.

    The fiber A (column-scaled) is factored by QR with column pivoting,
    A P = Q R.  Its numerical rank rho is the count of |R_kk| > theta |R_00|;
    the first rho pivot columns are kept and Q_rho (orthonormal, same span) is
    the basis maxvol works on: starting rows by elimination with partial
    pivoting on Q_rho, then maxvol over all rows.  The interpolation core is
    A_keep A_keep[I]^{-1} = Q_rho Q_rho[I]^{-1} (equal in exact arithmetic;
    the orthonormal form is the better-conditioned one).

    Returns (new index set, summed interpolant, interpolation core
    G as an (outer, N, rank) array)."""
    raw = _fiber(tensor, d, n, k, outer, cols, direction)
    diag.evaluations += raw.size
    a_mat = column_scaled(raw)
    q, r, _ = scipy.linalg.qr(a_mat, mode="economic", pivoting=True)
    rdiag = np.abs(np.diag(r))
    if rdiag.size == 0 or not (rdiag[0] > 0):
        raise FloatingPointError("fiber matrix has numerical rank 0")
    rho = int(np.count_nonzero(rdiag > opts.theta * rdiag[0]))
    basis = q[:, :rho]
    rows, _ = gepp_select(basis, 0.0)
    rows, swaps, ok = maxvol(basis, rows, opts.tau, opts.swap_cap * len(rows))
    diag.swaps += swaps
    diag.maxvol_unconverged += 0 if ok else 1
    g = basis @ np.linalg.inv(basis[rows, :])
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

def tt_cross_sum(tensor, r_max, seed, term=0, opts=None, keep_train=False, select=None):
    """TT-cross approximation of sum over the grid of ``tensor``; returns (sum, diag).

    With ``keep_train`` the cores of the latest left-to-right half-sweep are kept
    in ``diag.train``: G_0, ..., G_{d-2} (interpolation cores, (r_{k-1}, N, r_k))
    and the end core's fiber (r_{d-2}, N, 1); their product is the train whose
    weighted sum that half-sweep estimated.  ``select`` replaces the matrix cross
    step of one core (default ``core_select``; the tests' kernel-schedule replay
    passes its own)."""
    opts = opts or CrossOptions()
    select = select or core_select
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
                lsets[k + 1], gsum, core = select(tensor, d, n, k, lsets[k], rsets[k + 1], "lr", opts, diag)
                cores.append(core)
                v = v @ gsum
            est = complex(v @ core_sum(tensor, d, n, d - 1, lsets[d - 1], "lr", diag, cores))
            if keep_train:
                diag.train = cores
        else:
            v = np.ones(1, dtype=np.complex128)
            for k in range(d - 1, 0, -1):
                rsets[k], gsum, _ = select(tensor, d, n, k, rsets[k + 1], lsets[k], "rl", opts, diag)
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


def tt_price(problem, opts=None, select=None):
    """Price = Re(sum over terms of scale * TT-cross sum); returns (price, imag, diags)."""
    from .integrand import tensors_for

    acc = 0j
    diags = []
    for term, t in enumerate(tensors_for(problem)):
        est, dg = tt_cross_sum(t, int(problem.max_rank), int(problem.seed), term, opts, select=select)
        acc += t.scale * est
        diags.append(dg)
    return acc.real, acc.imag, diags


def dense_from_cores(cores):
    """Brute-force TT -> dense tensor (for pinning the contraction on tiny cases)."""
    out = cores[0]
    for c in cores[1:]:
        out = np.tensordot(out, c, axes=([-1], [0]))
    return out.reshape(out.shape[1:-1])
