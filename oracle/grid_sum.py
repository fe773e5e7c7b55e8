"""The exact N^d grid sum of the call on the minimum, for equicorrelated assets, at any d.

Test infrastructure only (see the package docstring).

What it computes.  The discretised price of Eq. (main) / Eq. (discr) on the
midpoint grid, V_N = Re{ e^{-rT} (eta/2 pi)^d sum_u phi_T(-z) vhat_min(z) },
z = u + i delta, summed over all N^d grid points u.  The full sum
(``integrand.full_grid_price``) is feasible only up to d = 4; this routine
reaches the same number at any d, so the TT-cross trains of the oracle and of
the CUDA path can be measured against the sum they approximate (their TT
error), not only against the exact integral (which adds the grid's own
discretisation error).

Derivation (textbook identities; the paper has no counterpart).  With
mu_j = ln S0_j + (r - sigma_j^2/2) T, the integrand at z = u + i delta is
    F(u) = C0 exp(-i u.a) exp(-T/2 u^T Cov u) / ((1 - sum delta + i sum u) prod_j (i u_j - delta_j)),
    C0 = (-1)^(d+1) K^(1 - sum delta) exp(delta.mu + T/2 delta^T Cov delta),
    a  = mu + T Cov delta - ln K,
(phi_T(w) = exp(i w.mu - T/2 w^T Cov w) at w = -z, and
vhat_min(z) = (-1)^(d+1) K^(1+i sum z)/((1+i sum z) prod (i z_j))).  Two
factors couple the axes, and each becomes a product of per-axis factors under
an integral:
  * equicorrelation Cov = D(rho 11^T + (1-rho) I)D, D = diag(sigma):
    u^T Cov u = rho s^2 + (1-rho) sum sigma_j^2 u_j^2 with s = sum sigma_j u_j,
    and exp(-T rho s^2 / 2) = E_Z[exp(i sqrt(T rho) s Z)], Z standard normal
    (the characteristic function of the normal law);
  * 1/(1 - sum delta + i sum u) = -int_0^inf exp(-t (sum delta - 1)) exp(i t sum u) dt,
    valid on the strip sum delta > 1.
Both hold exactly for every grid point, so
    sum_u F(u) = -C0 int_0^inf e^{-t (sum delta - 1)} E_Z[ prod_j h_j(Z, t) ] dt,
    h_j(Z, t) = sum_k exp(-T (1-rho) sigma_j^2 u_k^2 / 2) exp(-i u_k a_j)
                exp(i u_k (sqrt(T rho) sigma_j Z + t)) / (i u_k - delta_j).
The sums over k are exact; only the two one-dimensional integrals are
quadratures:
  * Z: trapezoid rule on [-z_max, z_max] with step h.  For a Gaussian-weighted
    integrand the rule is exact up to aliasing at the frequency 2 pi / h, and
    the integrand's frequencies in Z are at most sqrt(T rho) sum_j sigma_j L.
  * t: composite Gauss-Legendre on [0, t_max], panels short against the
    integrand's fastest oscillation in t (frequency at most d L), and
    t_max where exp(-t (sum delta - 1)) is below 1e-17.
The default steps resolve those frequencies with margin; a test halves them
and checks that the value does not move.

Pins (tests/test_oracle_grid_sum.py): equal to the brute-force full grid sum
at d = 1, 2, 3, 4 to ~1e-12; converges to the one-factor closed form as N
grows.
"""
from __future__ import annotations

import math

import numpy as np


def _gauss_legendre_panels(t_max, width, order):
    nodes, weights = np.polynomial.legendre.leggauss(order)
    npan = max(1, int(math.ceil(t_max / width)))
    w = t_max / npan
    left = np.arange(npan) * w
    t = (left[:, None] + 0.5 * w * (nodes[None, :] + 1.0)).ravel()
    tw = np.broadcast_to(0.5 * w * weights[None, :], (npan, order)).ravel()
    return t, tw


def grid_sum_min_call(spot, sigma, rho, rate, maturity, strike, damping, n_grid, trunc_L,
                      refine=1.0, order=8):
    """Exact midpoint-grid price of the call on the minimum (equicorrelated, rho >= 0).

    ``damping`` is alpha_j (Im z_j = delta_j = -alpha_j).  ``refine`` > 1 shrinks
    both quadrature steps by that factor (for the convergence check).  Returns
    (price, imaginary part); the imaginary part is zero up to the quadrature
    and rounding (the grid is symmetric).
    """
    spot = np.asarray(spot, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    delta = -np.asarray(damping, dtype=np.float64)
    d = spot.size
    if not (rho >= 0.0):
        raise ValueError("the one-factor decoupling needs rho >= 0")
    if np.any(delta <= 0) or delta.sum() <= 1.0:
        raise ValueError("damping outside the min-call strip")
    T, K = float(maturity), float(strike)
    cov = rho * np.outer(sigma, sigma) + (1.0 - rho) * np.diag(sigma ** 2)
    mu = np.log(spot) + (rate - 0.5 * sigma ** 2) * T
    cd = cov @ delta
    a = mu + T * cd - math.log(K)
    log_c0 = (1.0 - delta.sum()) * math.log(K) + delta @ mu + 0.5 * T * (delta @ cd)
    sign_c0 = -1.0 if d % 2 == 0 else 1.0           # (-1)^(d+1)
    eta = 2.0 * trunc_L / n_grid
    u = -trunc_L + (np.arange(n_grid) + 0.5) * eta
    excess = delta.sum() - 1.0

    # Z: trapezoid on a uniform grid
    omega_z = math.sqrt(T * rho) * sigma.sum() * trunc_L
    h = 2.0 * math.pi / (omega_z + 40.0) / refine
    z_max = 9.0
    nz = 2 * int(math.ceil(z_max / h)) + 1
    zs = np.linspace(-z_max, z_max, nz)
    zw = (zs[1] - zs[0]) * np.exp(-0.5 * zs ** 2) / math.sqrt(2.0 * math.pi)
    # t: Gauss-Legendre panels
    omega_t = d * trunc_L
    t_max = 40.0 / excess
    ts, tw = _gauss_legendre_panels(t_max, math.pi / (2.0 * omega_t) / refine, order)
    tw = tw * np.exp(-excess * ts)

    e_t = np.exp(1j * np.outer(u, ts))              # (N, nt): exp(i t u_k)
    prod = np.ones((nz, ts.size), dtype=np.complex128)
    for j in range(d):
        g = (np.exp(-0.5 * T * (1.0 - rho) * sigma[j] ** 2 * u ** 2 - 1j * u * a[j])
             / (1j * u - delta[j]))                  # (N,)
        gz = g[None, :] * np.exp(1j * math.sqrt(T * rho) * sigma[j] * np.outer(zs, u))  # (nz, N)
        prod *= gz @ e_t
    total = -(zw @ prod @ tw)                        # sum_u F(u) / C0
    val = sign_c0 * math.exp(log_c0) * total
    scale = math.exp(-rate * T) * (eta / (2.0 * math.pi)) ** d
    v = scale * val
    return float(v.real), float(v.imag)


def grid_sum_for(problem, refine=1.0):
    """``grid_sum_min_call`` for a Problem whose covariance is equicorrelated."""
    cov = np.asarray(problem.cov, dtype=np.float64)
    sigma = np.sqrt(np.diag(cov))
    corr = cov / np.outer(sigma, sigma)
    d = sigma.size
    off = corr[~np.eye(d, dtype=bool)]
    rho = float(off.mean()) if d > 1 else 0.0
    if d > 1 and np.max(np.abs(off - rho)) > 1e-12:
        raise ValueError("covariance is not equicorrelated")
    if problem.payoff != "min":
        raise ValueError("the one-factor grid sum covers the call on the minimum")
    return grid_sum_min_call(problem.spot, sigma, rho, problem.rate, problem.maturity, problem.strike,
                             problem.damping, problem.n_grid, problem.trunc_L, refine=refine)
