"""Exact partition function of the finite periodic L x L Ising ferromagnet.

Population annealing estimates the free energy through ln Z(beta_i) =
N ln 2 + sum_k ln Q_k (Sec. 5.4, Eq. (13)); the paper judges a Monte Carlo
simulation of the 2D Ising model against the exact finite-lattice energy
(the Ising application test of Sec. 4). This module supplies that exact value:
Kaufman's closed form for the partition function of an L x L torus
(B. Kaufman, Phys. Rev. 76, 1232 (1949); A. E. Ferdinand and M. E. Fisher,
Phys. Rev. 185, 832 (1969)), evaluated in log space with explicit signs:

  Z = 1/2 (2 sinh 2K)^(N/2) (Z1 + Z2 + Z3 + Z4),   K = beta J, N = L^2,
  Z1 = prod_{r=0}^{L-1} 2 cosh(L g_{2r+1} / 2),  Z2 = same with sinh,
  Z3 = prod_{r=0}^{L-1} 2 cosh(L g_{2r} / 2),    Z4 = same with sinh,
  cosh g_k = cosh 2K coth 2K - cos(pi k / L)  (k >= 1),
  g_0 = 2K + ln tanh K   (signed: negative above the critical temperature).

Pure Python floats (fp64); no dependency beyond ``math``.
"""
from __future__ import annotations

import math

BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))  # Onsager's critical coupling


def _log_2cosh(x: float) -> float:
    ax = abs(x)
    return ax + math.log1p(math.exp(-2.0 * ax))


def _log_abs_2sinh(x: float):
    """(ln|2 sinh x|, sign)."""
    if x == 0.0:
        return -math.inf, 0.0
    ax = abs(x)
    return ax + math.log1p(-math.exp(-2.0 * ax)), math.copysign(1.0, x)


def _gamma(k: int, K: float, L: int) -> float:
    if k == 0:
        return 2.0 * K + math.log(math.tanh(K))
    c = math.cosh(2.0 * K) / math.tanh(2.0 * K) - math.cos(math.pi * k / L)
    return math.acosh(c)


def ising2d_lnZ(L: int, beta: float, J: float = 1.0) -> float:
    """ln Z of the L x L periodic Ising model with coupling J at inverse temperature beta.

    beta = 0 gives N ln 2 exactly.
    """
    if L < 2:
        raise ValueError("L must be >= 2")
    N = L * L
    K = beta * J
    if K == 0.0:
        return N * math.log(2.0)
    if K < 0:
        raise ValueError("antiferromagnetic coupling not supported")
    logs = []
    # Z1, Z2: odd gammas
    l1 = 0.0
    l2, s2 = 0.0, 1.0
    for r in range(L):
        g = _gamma(2 * r + 1, K, L)
        l1 += _log_2cosh(L * g / 2.0)
        ls, sg = _log_abs_2sinh(L * g / 2.0)
        l2 += ls
        s2 *= sg
    l3 = 0.0
    l4, s4 = 0.0, 1.0
    for r in range(L):
        g = _gamma(2 * r, K, L)
        l3 += _log_2cosh(L * g / 2.0)
        ls, sg = _log_abs_2sinh(L * g / 2.0)
        l4 += ls
        s4 *= sg
    logs = [(l1, 1.0), (l2, s2), (l3, 1.0), (l4, s4)]
    lmax = max(l for l, s in logs if s != 0.0)
    acc = math.fsum(s * math.exp(l - lmax) for l, s in logs if s != 0.0)
    return -math.log(2.0) + 0.5 * N * math.log(2.0 * math.sinh(2.0 * K)) + lmax + math.log(acc)


def ising2d_lnZ_per_site(L: int, beta: float) -> float:
    return ising2d_lnZ(L, beta) / (L * L)


def ising2d_free_energy_per_site(L: int, beta: float) -> float:
    """f = -ln Z / (beta N) (units of J)."""
    return -ising2d_lnZ(L, beta) / (beta * L * L)


def ising2d_energy_per_site(L: int, beta: float, h: float = 1e-5) -> float:
    """u = -(1/N) d ln Z / d beta, by a fourth-order central difference."""
    N = L * L
    f = lambda b: ising2d_lnZ(L, b)
    d = (-f(beta + 2 * h) + 8 * f(beta + h) - 8 * f(beta - h) + f(beta - 2 * h)) / (12 * h)
    return -d / N


def onsager_lnZ_per_site_at_critical() -> float:
    """Thermodynamic-limit -beta f at the critical point: ln(2)/2 + 2G/pi."""
    catalan = 0.915965594177219015054603514932384110774
    return 0.5 * math.log(2.0) + 2.0 * catalan / math.pi
