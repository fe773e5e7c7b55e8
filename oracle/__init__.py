"""Plain FP64 CPU oracle for the tensor-train Fourier pricer (arXiv 2203.02804).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library, its
Python binding) imports, links or calls anything in this package; only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may use it.  It shares no code with the CUDA
path: the integrand is written straight from its definition (characteristic
function times payoff transform, Section III.C of the paper), the TT-cross
follows the matrix-cross / maxvol description of Section IV.B step by step,
and the closed forms are textbook results used as pins.

Modules
  integrand     -- the GBM characteristic function, payoff transforms,
                   the quadrature grid and the full N^d grid sum (Eq. main,
                   Eq. discr)
  closed_forms  -- Black-Scholes (Eq. BSexact), the two-asset Stulz formula,
                   one-factor semi-analytic prices, Monte Carlo (Eq. mc)
  ttcross       -- GEPP tournament + maxvol row selection and the TT-cross
                   sweeps that put the integrand into tensor-train form and
                   contract it with the quadrature weights (Section IV)
  splitmix      -- the SplitMix64 counter-based generator (Steele, Lea and
                   Flood 2014) used to draw the random initial pivots
  twomps        -- the paper's two-train (bra-ket) form: the payoff transform
                   and the characteristic function put into tensor-train form
                   separately, then contracted site by site (Eq. braket)
  mlp           -- the learned surrogate's network in FP64: fully connected
                   layers with SiLU, their backward pass, MSE and Adam
                   (Kingma and Ba 2015); no counterpart in the paper

Parity status of every function is stated in its docstring; no function here
is "parity unpinned": each is pinned by a test in tests/test_oracle_*.py
against a closed form, an identity, brute force, or Monte Carlo.
"""
