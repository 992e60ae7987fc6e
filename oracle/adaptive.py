"""Adaptive nonuniform selection probabilities (oracle; test infrastructure).

Sec. 4 of arXiv:1610.08895: c_i measures the relative distance of the block
residual to its ball, and p_i follows eq. (prob-choice):

    p_i = p_min + min((n - d p_min) c_i / sum_k c_k + a, p_max - p_min),

with a >= 0 the smallest value giving sum_i p_i = n (a = 0 unless some p_i
saturates at p_max), and p_i = n/d for all i when sum_k c_k = 0.

Reading of what the paper leaves open: a is found exactly. The left side
f(a) = sum_i min(q_i + a, cap) is continuous, piecewise linear and
non-decreasing, so the oracle walks its breakpoints in increasing order and
solves the linear piece that contains the target.
"""
import numpy as np


def residual_distance(res_norm, eps):
    """c_i = max(||Phi_i x - y_i|| - eps_i, 0)^2 / eps_i^2 (Sec. 4)."""
    res_norm = np.asarray(res_norm, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    return np.maximum(res_norm - eps, 0.0) ** 2 / eps ** 2


def probabilities(c, n, p_min, p_max):
    """Eq. (prob-choice) with the rebalancing offset a solved exactly."""
    c = np.asarray(c, dtype=np.float64)
    d = len(c)
    if not (p_min <= n / d and p_min <= p_max and p_max * d >= n):
        raise ValueError("need p_min <= n/d, p_min <= p_max and p_max >= n/d")
    total = c.sum()
    if total == 0.0:
        return np.full(d, n / d)
    q = (n - d * p_min) * c / total
    cap = p_max - p_min
    target = q.sum()                   # = n - d p_min
    if np.all(q <= cap):
        return p_min + q               # a = 0: no block saturates
    # f(a) = sum min(q_i + a, cap); block i saturates once a >= cap - q_i.
    brk = np.sort(np.maximum(cap - q, 0.0))
    a_lo = 0.0
    a = None
    for k in range(d + 1):
        a_hi = brk[k] if k < d else np.inf
        if a_hi < a_lo:
            continue
        sat = (cap - q) <= a_lo        # saturated throughout (a_lo, a_hi)
        n_free = np.count_nonzero(~sat)
        base = cap * np.count_nonzero(sat) + q[~sat].sum()
        # on this piece f(a) = base + n_free * a
        if n_free == 0:
            a = a_lo                   # every block saturated: f = d * cap >= target
            break
        cand = (target - base) / n_free
        if cand <= a_hi:
            a = max(cand, a_lo)
            break
        a_lo = a_hi
    if a is None:
        raise ValueError("no rebalancing offset reaches sum p = n")
    return p_min + np.minimum(q + a, cap)
