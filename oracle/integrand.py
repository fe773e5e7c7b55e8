"""The d-dimensional damped Fourier pricing integrand and its full grid sum.

Test infrastructure only (see the package docstring).  Everything here is the
plain definition written out in complex FP64 NumPy; nothing is factored,
log-scaled or reordered the way the CUDA path does it.

Paper passages followed
  * characteristic function of correlated GBM, Section III.C: with
    mu_j = ln S0_j + (r - sigma_j^2/2) T,
        phi_T(w) = exp(i w.mu - T/2 w^T Cov w).
    The paper's display omits the factor T on the quadratic term; T = 1 in all
    of its experiments.  The factor is restored here (pinned by the martingale
    identity phi(-i e_j) = S0_j e^{rT}).
  * min-call payoff transform, Section III.C (after Eberlein et al.):
        vhat_min(z) = (-1)^(d+1) K^(1 + i sum z) / ((1 + i sum z) prod_j (i z_j)),
    valid for Im z_j > 0 and sum_j Im z_j > 1.  The printed constant
    K^(..)/((-1)^d (1+i sum z) prod z_j) differs from this by i^d (-1); the form
    above is what integrating (min S - K)^+ = int_K^inf prod_j 1{S_j > s} ds
    gives, reduces to the single-asset transform at d = 1 as the paper says it
    should, and is pinned by Black-Scholes, Stulz and the one-factor formula.
  * the price as a damped Fourier integral, Eq. (main), with the d-dimensional
    normalisation (2 pi)^(-d) and the uniform grid sum of Eq. (discr) applied on
    every axis (weight eta per axis).
  * call on the maximum (not in the paper): split the payoff by which asset is
    the maximum, (max S - K)^+ = sum_j (S_j - K)^+ 1{S_j = max S}.  Term j in
    the variables y_j = x_j, y_l = x_l - x_j has the separable payoff
    (e^{y_j} - K)^+ prod_{l != j} 1{y_l <= 0}, whose transform is
        K^(1 + i z_j) / ((i z_j)(1 + i z_j)) * prod_{l != j} 1 / (i z_l)
    on Im z_j > 1, Im z_l < 0; Y = A_j X is Gaussian with mean A_j mu and
    covariance A_j Cov A_j^T, so its characteristic function has the same form.

Conventions (the readings used throughout the project)
  * damping: the caller's ``damping[j]`` is alpha_j in the workloads' sign
    convention (negative for the min-call); the imaginary shift is
    Im z_j = delta_j = -damping[j] for the min-call.  For the
    max-call term j, delta_j = 1 + |damping[j]| on the maximum's axis and
    delta_l = -|damping[l]| on the others (so the aliasing rate on every axis is
    |damping|, as for the min-call).
  * grid: N midpoints on [-L, L], u_k = -L + (k + 1/2) eta, eta = 2L/N.  The
    grid is symmetric, F(-u) = conj F(u), so the exact grid sum is real.
"""
from __future__ import annotations

import math

import numpy as np


# ----------------------------------------------------------------------------
# model pieces
# ----------------------------------------------------------------------------

def drift_mean(spot, cov, rate, maturity):
    """mu_j = ln S0_j + (r - Cov_jj / 2) T  (Section III.C, mu_j)."""
    spot = np.asarray(spot, dtype=np.float64)
    cov = np.asarray(cov, dtype=np.float64)
    return np.log(spot) + (rate - 0.5 * np.diag(cov)) * maturity


def char_fn(w, mu, cov, maturity):
    """phi_T(w) = exp(i w.mu - T/2 w^T Cov w) for complex w of shape (..., d)."""
    w = np.asarray(w, dtype=np.complex128)
    lin = w @ np.asarray(mu, dtype=np.complex128)
    quad = np.einsum("...j,jk,...k->...", w, np.asarray(cov, dtype=np.complex128), w)
    return np.exp(1j * lin - 0.5 * maturity * quad)


def payoff_transform_min(z, strike):
    """vhat_min(z) = (-1)^(d+1) K^(1+i sum z) / ((1+i sum z) prod(i z_j))."""
    z = np.asarray(z, dtype=np.complex128)
    d = z.shape[-1]
    sz = z.sum(axis=-1)
    kpow = np.exp((1.0 + 1j * sz) * math.log(strike))
    return (-1.0) ** (d + 1) * kpow / ((1.0 + 1j * sz) * np.prod(1j * z, axis=-1))


def payoff_transform_max_term(z, strike, j):
    """Transform of (e^{y_j} - K)^+ prod_{l != j} 1{y_l <= 0} (max-call term j)."""
    z = np.asarray(z, dtype=np.complex128)
    zj = z[..., j]
    val = np.exp((1.0 + 1j * zj) * math.log(strike)) / ((1j * zj) * (1.0 + 1j * zj))
    others = np.delete(z, j, axis=-1)
    if others.shape[-1]:
        val = val / np.prod(1j * others, axis=-1)
    return val


def max_term_transform_matrix(d, j):
    """A_j: y_j = x_j, y_l = x_l - x_j (unit determinant)."""
    a = np.eye(d)
    for l in range(d):
        if l != j:
            a[l, j] = -1.0
    return a


# ----------------------------------------------------------------------------
# grid and damping readings
# ----------------------------------------------------------------------------

def grid(n_grid, trunc_l):
    """Midpoint grid u_k = -L + (k + 1/2) eta on [-L, L], eta = 2L/N."""
    eta = 2.0 * trunc_l / n_grid
    return -trunc_l + (np.arange(n_grid) + 0.5) * eta, eta


def min_call_shift(damping):
    """delta_j = -damping_j; the strip needs delta_j > 0 and sum delta > 1."""
    delta = -np.asarray(damping, dtype=np.float64)
    return delta


def max_call_shift(damping, j):
    """delta for max-call term j: 1 + |a_j| on axis j, -|a_l| elsewhere."""
    a = np.abs(np.asarray(damping, dtype=np.float64))
    delta = -a.copy()
    delta[j] = 1.0 + a[j]
    return delta


# ----------------------------------------------------------------------------
# the tensors TT-cross approximates
# ----------------------------------------------------------------------------

class FourierTensor:
    """T[i_1..i_d] = phi(-z) vhat(z) at z = u_i + i delta, on the N^d grid.

    ``term`` is None for the min-call, or j for term j of the max-call.
    ``scale`` = e^{-rT} (eta / 2 pi)^d, so that price = Re(scale * sum T).
    """

    def __init__(self, problem, term=None):
        self.p = problem
        self.d = len(problem.spot)
        self.n = int(problem.n_grid)
        self.u, self.eta = grid(self.n, float(problem.trunc_L))
        mu = drift_mean(problem.spot, problem.cov, problem.rate, problem.maturity)
        cov = np.asarray(problem.cov, dtype=np.float64)
        self.term = term
        if term is None:
            self.delta = min_call_shift(problem.damping)
            self.mu, self.cov = mu, cov
        else:
            a = max_term_transform_matrix(self.d, term)
            self.delta = max_call_shift(problem.damping, term)
            self.mu, self.cov = a @ mu, a @ cov @ a.T
        self.scale = math.exp(-problem.rate * problem.maturity) * (self.eta / (2 * math.pi)) ** self.d
        # spread of TT-cross's random initial pivots (grid steps per axis)
        from .ttcross import pivot_widths
        self.pivot_widths = pivot_widths(np.diag(self.cov), float(problem.maturity), self.eta)

    def at_points(self, u):
        """Integrand at real points u of shape (..., d)."""
        z = np.asarray(u, dtype=np.float64) + 1j * self.delta
        phi = char_fn(-z, self.mu, self.cov, self.p.maturity)
        if self.term is None:
            v = payoff_transform_min(z, self.p.strike)
        else:
            v = payoff_transform_max_term(z, self.p.strike, self.term)
        return phi * v

    def __call__(self, idx):
        """Entries at integer multi-indices idx of shape (..., d)."""
        return self.at_points(self.u[np.asarray(idx)])


def tensors_for(problem):
    """The list of tensors whose scaled sums add up to the price."""
    if problem.payoff == "min":
        return [FourierTensor(problem)]
    if problem.payoff == "max":
        return [FourierTensor(problem, term=j) for j in range(len(problem.spot))]
    raise ValueError(f"unknown payoff {problem.payoff!r}")


# ----------------------------------------------------------------------------
# full grid sum (Eq. discr on every axis; feasible for small N^d)
# ----------------------------------------------------------------------------

def full_grid_sum(tensor, chunk=1 << 18):
    """Exact sum of the tensor over its N^d grid (pairwise within chunks, fsum across)."""
    d, n = tensor.d, tensor.n
    total = n ** d
    re_parts, im_parts = [], []
    for start in range(0, total, chunk):
        flat = np.arange(start, min(total, start + chunk), dtype=np.int64)
        idx = np.empty((flat.size, d), dtype=np.int64)
        rem = flat
        for ax in range(d - 1, -1, -1):
            idx[:, ax] = rem % n
            rem = rem // n
        vals = tensor(idx)
        s = vals.sum()
        re_parts.append(s.real)
        im_parts.append(s.imag)
    return complex(math.fsum(re_parts), math.fsum(im_parts))


def full_grid_price(problem):
    """Price by the full N^d grid sum: Re(sum over terms of scale * sum T).

    Returns (price, imaginary part) -- the imaginary part is zero up to rounding
    because the midpoint grid is symmetric.
    """
    acc = 0j
    for t in tensors_for(problem):
        acc += t.scale * full_grid_sum(t)
    return acc.real, acc.imag
