"""Detection probability of a rough estimator (Section 3.2, Eq. 2-5) — TEST INFRASTRUCTURE ONLY.

A rough estimator RE of eta cells records a destination only when its hash H1 has
LSB >= tau (probability 2^-tau), in the cell chosen by H2. For a host with n distinct
destinations:

* FN(alpha, eta): the number of ways to throw alpha distinct balls into eta boxes with no
  box empty, by the paper's recursion (the Lemma of Section 3.2): all eta^alpha throws
  minus those that leave some box empty, FN(alpha, 1) = 1.
* Eq. 2: Pr{alpha, eta, eta1} = C(eta, eta1) * FN(alpha, eta1) / eta^alpha, the chance that
  alpha recorded destinations set exactly eta1 cells (the Theorem of Section 3.2).
* Eq. 3: Pr{n, alpha} = C(n, alpha) p^alpha (1 - p)^(n - alpha), p = 2^-tau, the chance
  that alpha of the n destinations are recorded.
* Eq. 4: Pr{n, eta, tau, eta1} = sum over alpha of Eq. 3 times Eq. 2.
* Eq. 5: Pr+{n, eta, tau, m} = sum over eta1 >= m of Eq. 4, the chance that at least m
  cells are set, i.e. that the estimator reports the host (m = ceil(rho * eta)).

Exact integers for the counts; the binomial weights in FP64 through log-gamma. Pinned by
tests against brute-force enumeration, the inclusion-exclusion closed form for
surjections, normalisation, and Monte-Carlo runs of the oracle's own estimator.
"""
from __future__ import annotations

import math
from functools import lru_cache


@lru_cache(maxsize=None)
def surjections(alpha: int, eta: int) -> int:
    """FN(alpha, eta) by the recursion FN = eta^alpha - sum_{i=1}^{eta-1} C(eta, i) FN(alpha, i)."""
    if eta < 1 or alpha < eta:
        return 0
    if eta == 1:
        return 1
    total = eta ** alpha
    for i in range(1, eta):
        total -= math.comb(eta, i) * surjections(alpha, i)
    return total


def pr_cells_set(alpha: int, eta: int, eta1: int) -> float:
    """Eq. 2: probability that alpha recorded destinations set exactly eta1 of eta cells."""
    if alpha == 0:
        return 1.0 if eta1 == 0 else 0.0
    if eta1 < 1 or eta1 > eta or eta1 > alpha:
        return 0.0
    return (math.comb(eta, eta1) * surjections(alpha, eta1)) / (eta ** alpha)


def pr_recorded(n: int, alpha: int, tau: int) -> float:
    """Eq. 3: probability that alpha of the host's n destinations pass the sampling."""
    if alpha < 0 or alpha > n:
        return 0.0
    p = 2.0 ** (-tau)
    if p == 1.0:
        return 1.0 if alpha == n else 0.0
    log = (math.lgamma(n + 1) - math.lgamma(alpha + 1) - math.lgamma(n - alpha + 1)
           + alpha * math.log(p) + (n - alpha) * math.log1p(-p))
    return math.exp(log)


def pr_cells_after_scan(n: int, eta: int, tau: int, eta1: int, alpha_max: int | None = None) -> float:
    """Eq. 4: probability that eta1 cells are set after the host's n destinations.
    alpha_max bounds the sum (terms beyond it are below 1e-300 for the sizes used)."""
    top = n if alpha_max is None else min(n, alpha_max)
    return sum(pr_recorded(n, a, tau) * pr_cells_set(a, eta, eta1) for a in range(eta1, top + 1))


def pr_reported(n: int, eta: int, tau: int, m: int, alpha_max: int | None = None) -> float:
    """Eq. 5: probability that at least m cells are set, i.e. the host is reported hot."""
    return sum(pr_cells_after_scan(n, eta, tau, e, alpha_max) for e in range(m, eta + 1))
