"""Adaptive temperature steps for population annealing: the oracle side.

TEST INFRASTRUCTURE (see oracle/__init__.py): used only by tests, smoke() and
bench.py's baseline legs; shares no code with the CUDA library.

Sec. 5.4 cites adaptive temperature steps without specifying them. The
reading used here: the next step dbeta is chosen so that the energy histogram
of the current population, h(E), and the same histogram reweighted to
beta + dbeta, P1(E) proportional to h(E) exp(-dbeta E), overlap by a target
amount,

    alpha(dbeta) = sum_E min(P0(E), P1(E)),   P0 = h / R,

found by bisection (the resampling weights of Eq. (13) are exactly these
reweighting factors, so low overlap means few replicas carry the next
population). alpha(0) = 1 and alpha decreases towards P0(E_min).
Everything is fp64, plain numpy, in the order of the definition.
"""
from __future__ import annotations

import math

import numpy as np

BISECT_ITERS = 50


def histogram(E):
    """Energy levels in increasing order and their counts."""
    levels, counts = np.unique(np.asarray(E, dtype=np.int64), return_counts=True)
    return levels, counts.astype(np.float64)


def overlap(levels, counts, dbeta: float) -> float:
    R = counts.sum()
    p0 = counts / R
    w = counts * np.exp(-dbeta * (levels - levels[0]).astype(np.float64))
    p1 = w / w.sum()
    return float(np.minimum(p0, p1).sum())


def bisect_dbeta(levels, counts, target: float, dbeta_max: float):
    """Largest dbeta in [0, dbeta_max] with alpha(dbeta) >= target, to the
    resolution of BISECT_ITERS halvings: returns (dbeta, clamped) where
    clamped means alpha(dbeta_max) >= target and dbeta = dbeta_max."""
    if overlap(levels, counts, dbeta_max) >= target:
        return dbeta_max, True
    lo, hi = 0.0, dbeta_max
    for _ in range(BISECT_ITERS):
        mid = 0.5 * (lo + hi)
        if overlap(levels, counts, mid) >= target:
            lo = mid
        else:
            hi = mid
    return lo, False


def moments(levels, counts):
    """Population mean, variance and skewness of E (fp64)."""
    R = counts.sum()
    x = (levels - levels[0]).astype(np.float64)
    m1 = float((counts * x).sum() / R)
    d = x - m1
    var = float((counts * d * d).sum() / R)
    m3 = float((counts * d * d * d).sum() / R)
    skew = m3 / var ** 1.5 if var > 0 else 0.0
    return float(levels[0]) + m1, var, skew


def features(levels, counts, beta: float, L: int, R: int, N: int) -> np.ndarray:
    """MLP inputs: energy per spin, log(Var(E)/N + 1e-6), skewness (clipped to
    [-10, 10]), beta, log L, log R."""
    mean, var, skew = moments(levels, counts)
    return np.array([mean / N, math.log(var / N + 1e-6), max(-10.0, min(10.0, skew)), beta,
                     math.log(L), math.log(R)], dtype=np.float64)


def dbeta_from_output(y: float, var: float, dbeta_max: float) -> float:
    """MLP output y = log(dbeta * sigma_E) -> dbeta, capped at dbeta_max."""
    sigma = math.sqrt(max(var, 1e-12))
    return min(dbeta_max, math.exp(y) / sigma)


def target_from_dbeta(dbeta: float, var: float) -> float:
    return math.log(dbeta * math.sqrt(max(var, 1e-12)))


def choose_step(levels, counts, beta, L, R, N, dmax, target, params=None, lo=0.0, hi=1.0):
    """One adaptive step: the MLP proposal (if params are given) kept when its
    overlap lies in [lo, hi], else the bisection. Returns a dict with dbeta,
    alpha, kind (1 bisection, 2 proposal), proposal, alpha_proposal, evals."""
    from oracle import mlp

    out = dict(proposal=0.0, alpha_proposal=0.0, evals=0)
    _, var, _ = moments(levels, counts)
    if params is not None:
        x = features(levels, counts, beta, L, R, N)[None, :]
        y, _ = mlp.forward(mlp.bf16_round(params), x)
        prop = dbeta_from_output(float(y[0]), var, dmax)
        a = overlap(levels, counts, prop)
        out.update(proposal=prop, alpha_proposal=a, evals=1)
        if lo <= a <= hi:
            out.update(dbeta=prop, alpha=a, kind=2)
            return out
    d, clamped = bisect_dbeta(levels, counts, target, dmax)
    out.update(dbeta=d, alpha=overlap(levels, counts, d), kind=1,
               evals=out["evals"] + (1 if clamped else 1 + BISECT_ITERS))
    return out
