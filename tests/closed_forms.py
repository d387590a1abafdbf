"""Independent closed forms and brute force used to pin the oracle.

Nothing here is imported by the library.  Each routine is a different
algorithm from the oracle's backward induction:

* Black-Scholes-Merton prices with a continuous yield (textbook closed form);
* European lattice sums: the binomial and trinomial expectations of the payoff
  at expiry, summed term by term in log space;
* brute-force valuation on the NON-recombining tree (every path enumerated),
  which checks the lattice indexing and recombination of the oracle.
"""
from __future__ import annotations

import math
from typing import Sequence


def norm_cdf(x: float) -> float:
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def bs_call(S, K, r, q, sigma, E):
    d1 = (math.log(S / K) + (r - q + 0.5 * sigma * sigma) * E) / (sigma * math.sqrt(E))
    d2 = d1 - sigma * math.sqrt(E)
    return S * math.exp(-q * E) * norm_cdf(d1) - K * math.exp(-r * E) * norm_cdf(d2)


def bs_put(S, K, r, q, sigma, E):
    d1 = (math.log(S / K) + (r - q + 0.5 * sigma * sigma) * E) / (sigma * math.sqrt(E))
    d2 = d1 - sigma * math.sqrt(E)
    return K * math.exp(-r * E) * norm_cdf(-d2) - S * math.exp(-q * E) * norm_cdf(-d1)


def _log_sum(terms: Sequence[float]) -> float:
    return math.fsum(terms)


def binomial_european_call(S, K, T, u, p, m):
    """sum_j C(T,j) p^j (1-p)^(T-j) m^T (S u^(2j-T) - K)^+ in log space."""
    out = []
    lp, lq = math.log(p), math.log1p(-p)
    lT = math.lgamma(T + 1)
    for j in range(T + 1):
        pay = S * u ** (2 * j - T) - K
        if pay <= 0:
            continue
        lw = lT - math.lgamma(j + 1) - math.lgamma(T - j + 1) + j * lp + (T - j) * lq + T * math.log(m)
        out.append(math.exp(lw) * pay)
    return _log_sum(out)


def trinomial_european_call(S, K, T, u, pu, po, pd, m):
    """sum over (n_u, n_o, n_d) of the multinomial weight times
    m^T (S u^(n_u - n_d) - K)^+."""
    out = []
    lT = math.lgamma(T + 1)
    lu, lo, ld = math.log(pu), math.log(po), math.log(pd)
    for nu in range(T + 1):
        for nd in range(T + 1 - nu):
            pay = S * u ** (nu - nd) - K
            if pay <= 0:
                continue
            no = T - nu - nd
            lw = (lT - math.lgamma(nu + 1) - math.lgamma(no + 1) - math.lgamma(nd + 1)
                  + nu * lu + no * lo + nd * ld + T * math.log(m))
            out.append(math.exp(lw) * pay)
    return _log_sum(out)


def brute_force_tree(level_max: int, steps, exercise, x0, american=True):
    """Value an option on the non-recombining tree.

    ``steps`` is a list of (weight, move) pairs: the child state is
    ``x + move`` and its value is weighted by ``weight`` (weights already
    include discounting).  ``exercise(level, x)`` is the exercise value of a
    node; at the last level the value is max(exercise, 0).  Every path is
    enumerated separately (no recombination), so the cost is len(steps)^T.
    """
    def value(level, x):
        if level == level_max:
            return max(exercise(level, x), 0.0)
        cont = 0.0
        for w, mv in steps:
            cont += w * value(level + 1, x + mv)
        if american:
            return max(cont, exercise(level, x))
        return cont
    return value(0, x0)


def binomial_european_put(S, K, T, u, p, m):
    """sum_j C(T,j) p^j (1-p)^(T-j) m^T (K - S u^(2j-T))^+ in log space."""
    out = []
    lp, lq = math.log(p), math.log1p(-p)
    lT = math.lgamma(T + 1)
    for j in range(T + 1):
        pay = K - S * u ** (2 * j - T)
        if pay <= 0:
            continue
        lw = lT - math.lgamma(j + 1) - math.lgamma(T - j + 1) + j * lp + (T - j) * lq + T * math.log(m)
        out.append(math.exp(lw) * pay)
    return _log_sum(out)


def trinomial_european_put(S, K, T, u, pu, po, pd, m):
    """The multinomial expectation of m^T (K - S u^(n_u - n_d))^+."""
    out = []
    lT = math.lgamma(T + 1)
    lu, lo, ld = math.log(pu), math.log(po), math.log(pd)
    for nu in range(T + 1):
        for nd in range(T + 1 - nu):
            pay = K - S * u ** (nu - nd)
            if pay <= 0:
                continue
            no = T - nu - nd
            lw = (lT - math.lgamma(nu + 1) - math.lgamma(no + 1) - math.lgamma(nd + 1)
                  + nu * lu + no * lo + nd * ld + T * math.log(m))
            out.append(math.exp(lw) * pay)
    return _log_sum(out)


def norm_pdf(x: float) -> float:
    return math.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def bs_greeks(S, K, r, q, sigma, E, call=True):
    """Black-Scholes-Merton delta, gamma and theta (dV/dt in calendar time,
    per year) of a European call or put with continuous yield q."""
    sq = sigma * math.sqrt(E)
    d1 = (math.log(S / K) + (r - q + 0.5 * sigma * sigma) * E) / sq
    d2 = d1 - sq
    dq, dr = math.exp(-q * E), math.exp(-r * E)
    gamma = dq * norm_pdf(d1) / (S * sq)
    decay = -S * dq * norm_pdf(d1) * sigma / (2.0 * math.sqrt(E))
    if call:
        return (dq * norm_cdf(d1), gamma,
                decay - r * K * dr * norm_cdf(d2) + q * S * dq * norm_cdf(d1))
    return (-dq * norm_cdf(-d1), gamma,
            decay + r * K * dr * norm_cdf(-d2) - q * S * dq * norm_cdf(-d1))
