"""The paper's two-train (bra-ket) form of the price, in FP64.

Test infrastructure only (see the package docstring).

What the paper fixes (Section IV, Eq. braket; Section IV.A)
  * The price is e^{-rT} (2 pi)^{-d} times the inner product of two vectors on
    the N^d grid: one holds the payoff transform vhat(z), the other the
    characteristic function phi_T(-z), both at z = u + i delta.  Each vector is
    put into matrix-product (tensor-train) form by TT-cross separately, with
    its own bond dimension (D_v and D_phi in the paper's table), and the two
    trains are contracted site by site.

Readings
  * The bracket is the plain bilinear sum over the grid, sum_u vhat(z)
    phi_T(-z), without complex conjugation: that sum is what the pricing
    integral (Eq. main) discretises, and it is the product integrand the
    single-train path sums.  The grid weights (eta per axis) are folded into
    the tensor's scale as there.
  * Call on the maximum: each term j of the argmax split (see ``integrand``)
    is a bracket of its own pair of vectors, in the variables y = A_j x.
  * Stop rule.  The paper sizes the bond dimensions so that one sweep
    converges, judged by sampled pointwise error (Section IV.B), not by the
    sum.  A factor's own grid sum is no guide here: the payoff transform's
    sum is ~1e-10 of its entries, so the single-train rule (two consecutive
    sums agreeing) never fires.  Each factor's cross therefore runs a fixed
    3 half-sweeps, left-to-right, right-to-left, left-to-right, and the train
    is the cores of the last one, built on right index sets the
    right-to-left half-sweep improved (``ttcross.tt_cross_sum(...,
    keep_train=True)``).  Elsewhere the options, seed and pivot rules are the
    single-train path's.  Both vectors use one rank cap, the problem's
    ``max_rank``.
  * The cross never raises a bond's rank once it falls.  Random right index
    sets that make a fiber rank-deficient (for the payoff transform, columns
    whose coordinate sums coincide give collinear columns) lower that bond
    for good.  Exactness at full rank therefore holds where the initial right
    sets are exhaustive (d = 2).
  * Site-by-site contraction: E_0 = [1]; E_k = sum_i G^v_k[:, i, :]^T E_{k-1}
    G^phi_k[:, i, :]; the bracket is the single entry of E_d.

Pins (tests/test_oracle_twomps.py): the contraction against the dense sum of
two small random trains built out by brute force; the two factors' product
against the single-train integrand; the full-rank bracket against the full
grid sum; the rank-1 train of the characteristic function without correlation
against the product of one-dimensional sums; the d=2 min-call and max-call prices
against Stulz's closed forms; the paper's d=3, 4 setting against the full grid sum.
"""
from __future__ import annotations

import math
from dataclasses import replace

import numpy as np

from .integrand import (FourierTensor, char_fn, payoff_transform_max_term, payoff_transform_min)
from .ttcross import CrossOptions, tt_cross_sum


class FactorTensor(FourierTensor):
    """One factor of the integrand on the grid: ``factor`` = "phi" gives
    phi_T(-z), "vhat" the payoff transform vhat(z) (min-call, or term j of the
    max-call).  Grid, shift, scale and initial-pivot spread are the product
    tensor's."""

    def __init__(self, problem, factor, term=None):
        super().__init__(problem, term)
        if factor not in ("phi", "vhat"):
            raise ValueError(f"unknown factor {factor!r}")
        self.factor = factor

    def at_points(self, u):
        z = np.asarray(u, dtype=np.float64) + 1j * self.delta
        if self.factor == "phi":
            return char_fn(-z, self.mu, self.cov, self.p.maturity)
        if self.term is None:
            return payoff_transform_min(z, self.p.strike)
        return payoff_transform_max_term(z, self.p.strike, self.term)


def mps_bracket(cores_a, cores_b):
    """sum_u A(u) B(u) for two tensor trains given by their cores (r_{k-1}, N, r_k),
    contracted site by site: E <- sum_i A_k[:, i, :]^T E B_k[:, i, :]."""
    if len(cores_a) != len(cores_b):
        raise ValueError("trains of different length")
    e = np.ones((1, 1), dtype=np.complex128)
    for ga, gb in zip(cores_a, cores_b):
        e = np.einsum("aib,ac,cid->bd", ga, e, gb)
    return complex(e[0, 0])


HALF_SWEEPS = 3


def two_train_options(opts=None):
    """The cross options of a factor train: those given (or the defaults) with a
    fixed count of half-sweeps (``HALF_SWEEPS`` unless given) and no early stop."""
    opts = opts or CrossOptions(max_half_sweeps=HALF_SWEEPS)
    return replace(opts, sweep_tol=0.0)


def factor_trains(problem, term=None, opts=None, select=None, rank_v=None, rank_phi=None):
    """TT-cross trains of vhat and phi for the min-call (term None) or max-call
    term j; returns (train_vhat, train_phi, diag_vhat, diag_phi).  The bond
    dimensions D_v and D_phi (the paper's table gives them separately) default
    to the problem's rank cap."""
    opts = two_train_options(opts)
    t_term = 0 if term is None else term
    caps = {"vhat": rank_v or int(problem.max_rank), "phi": rank_phi or int(problem.max_rank)}
    out = []
    for factor in ("vhat", "phi"):
        t = FactorTensor(problem, factor, term)
        _, dg = tt_cross_sum(t, caps[factor], int(problem.seed), t_term, opts, keep_train=True, select=select)
        out.append((dg.train, dg))
    return out[0][0], out[1][0], out[0][1], out[1][1]


def two_train_price(problem, opts=None, select=None, rank_v=None, rank_phi=None):
    """Price = Re(sum over terms of scale * <vhat | phi>); returns (price, imag, diags).
    ``select`` replaces the matrix cross step (default: the paper-order one)."""
    terms = [None] if problem.payoff == "min" else list(range(len(problem.spot)))
    acc = 0j
    diags = []
    for term in terms:
        tv, tp, dv, dp = factor_trains(problem, term, opts, select, rank_v, rank_phi)
        scale = FactorTensor(problem, "phi", term).scale
        acc += scale * mps_bracket(tv, tp)
        diags.append((dv, dp))
    return acc.real, acc.imag, diags


def separable_phi_sum(problem):
    """sum over the grid of phi_T(-z) when Cov is diagonal: the product over axes of
    one-dimensional sums (the closed form that pins the phi train)."""
    t = FactorTensor(problem, "phi")
    if np.count_nonzero(t.cov - np.diag(np.diag(t.cov))):
        raise ValueError("covariance is not diagonal")
    total = 1.0 + 0j
    for j in range(t.d):
        z = t.u + 1j * t.delta[j]
        # phi_T(-z) on axis j alone: exp(-i z mu_j - T/2 Cov_jj z^2)
        total *= np.sum(np.exp(-1j * z * t.mu[j] - 0.5 * t.p.maturity * t.cov[j, j] * z * z))
    return complex(total)
