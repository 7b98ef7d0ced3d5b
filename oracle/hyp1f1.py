"""The restricted confluent hypergeometric function of Appendix A.

G(a, b, r) = Gamma(a)/Gamma(b) exp(-c r^2) 1F1(a; b; z),   z = c^2 r^2 / (c + d),
with a = (n + l + 3)/2 and b = l + 3/2 in the GTO radial integral.

Two evaluations, each carrying the factor exp(-c r^2) inside so that nothing overflows:

* the power series of 1F1, term by term, starting from Gamma(a)/Gamma(b) exp(-c r^2);
* the large-z asymptotic series, 1F1 ~ exp(z) z^(a-b) Gamma(b)/Gamma(a) sum_s (b-a)_s (1-a)_s / s! z^-s, which
  turns into G = exp(z - c r^2) z^(a-b) sum_s ... and z - c r^2 < 0.

Which form is used at a given z follows a switch point that is found once per (a, b) by bisection. Reading (the
paper does not give the criterion): the switch is the smallest z in [1, 300] at which the asymptotic series,
truncated at its smallest term, agrees with the power series to 1e-13 relative; if it never does, the power
series is used everywhere.

Also here: the two-step downward recurrence in (a, b) and dG/dr = 2 c^2 r/(c+d) G(a+1, b+1) - 2 c r G(a, b).
"""
from __future__ import annotations

from functools import lru_cache
from math import lgamma

import numpy as np

_EPS = 1e-17


def series_scaled(a: float, b: float, z, log_scale):
    """Gamma(a)/Gamma(b) exp(log_scale) 1F1(a;b;z) by the power series (z >= 0), vectorised over z."""
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    log_scale = np.broadcast_to(np.asarray(log_scale, dtype=np.float64), z.shape)
    term = np.exp(lgamma(a) - lgamma(b) + log_scale)
    total = term.copy()
    s = 0
    active = np.ones(z.shape, dtype=bool)
    while np.any(active):
        term = np.where(active, term * (a + s) * z / ((b + s) * (s + 1.0)), 0.0)
        total = total + term
        s += 1
        # terms grow while (a+s) z > (b+s)(s+1); stop only once they shrink below eps of the sum
        shrinking = (a + s) * z < (b + s) * (s + 1.0)
        active = active & ~(shrinking & (term <= _EPS * total))
        if s > 100000:
            raise RuntimeError("1F1 series did not converge")
    return total


def asymptotic_scaled(a: float, b: float, z, log_scale):
    """exp(z + log_scale) z^(a-b) sum_s (b-a)_s (1-a)_s / s! z^-s, truncated at its smallest term (z > 0).

    Returns (value, last_term_ratio): the ratio |last kept term / sum| tells how accurate the truncation is.
    """
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    log_scale = np.broadcast_to(np.asarray(log_scale, dtype=np.float64), z.shape)
    term = np.ones_like(z)
    total = np.ones_like(z)
    last = np.ones_like(z)
    active = np.ones(z.shape, dtype=bool)
    s = 0
    while np.any(active) and s < 400:
        nxt = term * (b - a + s) * (1.0 - a + s) / ((s + 1.0) * z)
        # stop when the series terminates, when terms start to grow, or when converged
        grow = np.abs(nxt) >= np.abs(term)
        done = (nxt == 0.0) | grow
        upd = active & ~done
        total = np.where(upd, total + nxt, total)
        last = np.where(upd, np.abs(nxt), np.where(active & (nxt == 0.0), 0.0, last))
        term = np.where(upd, nxt, term)
        active = upd & (np.abs(nxt) > _EPS * np.abs(total))
        s += 1
    value = np.exp(z + log_scale + (a - b) * np.log(z)) * total
    return value, last / np.abs(total)


@lru_cache(maxsize=None)
def switch_point(a: float, b: float, tol: float = 1e-13) -> float:
    """Smallest z in [1, 300] from which the asymptotic form matches the series to tol (bisection); inf if none."""

    def ok(z: float) -> bool:
        ser = series_scaled(a, b, z, -z)[0]
        asy, _ = asymptotic_scaled(a, b, z, -z)
        return abs(asy[0] - ser) <= tol * abs(ser)

    lo, hi = 1.0, 300.0
    if not ok(hi):
        return float("inf")
    if ok(lo):
        return lo
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if ok(mid):
            hi = mid
        else:
            lo = mid
    return hi


def G(a: float, b: float, c: float, d: float, r) -> np.ndarray:
    """G(a, b, r) of Appendix A for arrays of r >= 0, using the series below the switch point, asymptotic above."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    z = c * c * r * r / (c + d)
    cr2 = c * r * r
    zs = switch_point(float(a), float(b))
    out = np.empty_like(r)
    lo = z < zs
    if np.any(lo):
        out[lo] = series_scaled(a, b, z[lo], -cr2[lo])
    if np.any(~lo):
        out[~lo] = asymptotic_scaled(a, b, z[~lo], -cr2[~lo])[0]
    return out


def dG_dr(a: float, b: float, c: float, d: float, r) -> np.ndarray:
    """dG/dr = 2 c^2 r / (c + d) G(a+1, b+1, r) - 2 c r G(a, b, r)   (Appendix A)."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    return 2.0 * c * c * r / (c + d) * G(a + 1.0, b + 1.0, c, d, r) - 2.0 * c * r * G(a, b, c, d, r)


def recurrence_step_ab(Ga1b2, Ga1b1, a: float, b: float, z):
    """G(a, b) = z (a - b)/a G(a+1, b+2) + b/a G(a+1, b+1)   (second relation of Eq. 1f1-recurrence)."""
    return z * (a - b) / a * Ga1b2 + b / a * Ga1b1


def recurrence_step_a1b1(Ga2b3, Ga1b2, b: float, z):
    """G(a+1, b+1) = z G(a+2, b+3) + (b + 1) G(a+1, b+2)   (first relation of Eq. 1f1-recurrence)."""
    return z * Ga2b3 + (b + 1.0) * Ga1b2
