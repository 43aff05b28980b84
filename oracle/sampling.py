"""Random variates from Philox words (oracle; test infrastructure only).

The paper fixes only that connection rules draw sources, weights and delays from
pseudo-random numbers (Methods, "Creation of the remote connection structures for
point-to-point MPI communication") following the rule conventions of Senk et al.
(2022).  The variates below are the build's readings of those draws:

* ``uniform_index``: integer in [0, n) as the high word of w * n (Lemire's
  multiply-shift, no rejection); integer-exact, so sources are bit-exact.
* ``u01``: ((w >> 9) + 0.5) * 2^-23, exact in fp32 and fp64 (24 significant
  bits), never 0 or 1.
* ``box_muller``: z = sqrt(-2 ln u1) cos(2 pi u2) (Box & Muller 1958).
* ``quantised_normal_table``: delay steps round(max(d, lo) / h), d ~ N(mu, sd),
  at least 1 step, drawn by inversion of an integer CDF table so that the decision is
  integer-only.  thr_s = floor(P(step <= s) 2^32 + 1/2); step = s_min + #{thr <= w}.
* ``poisson_table``: the same integer inversion for Poisson(lambda) counts.

Pinned by tests/test_oracle_sampling.py (closed-form probabilities, chi-square,
special cases).
"""
from __future__ import annotations

import math

import numpy as np

TWO32 = 4294967296.0
MAX_DELAY_STEPS = 255


def uniform_index(w, n: int):
    """Integer in [0, n) from a 32-bit word: floor(w * n / 2^32)."""
    return (np.asarray(w, dtype=np.uint64) * np.uint64(n)) >> np.uint64(32)


def u01(w):
    """Uniform in (0, 1) from the top 23 bits of a word, exact in fp32."""
    return ((np.asarray(w, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def box_muller(w2, w3):
    """Standard normal from two words (Box & Muller 1958), fp64."""
    u1, u2 = u01(w2), u01(w3)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def weight_values(dist, w2, w3, count: int):
    """Weights in fp64 for ``dist`` ('const' or 'normal_sign').  'normal_sign' draws
    mean + sd * z and clamps to 0 so the sign of the mean is kept (reading of
    "clipped to keep sign": clamp, not redraw, so the counter map stays fixed)."""
    if dist.kind == "const":
        return np.full(count, float(dist.mean))
    if dist.kind == "normal_sign":
        w = float(dist.mean) + float(dist.sd) * box_muller(w2, w3)
        return np.maximum(w, 0.0) if dist.mean >= 0 else np.minimum(w, 0.0)
    raise ValueError(dist.kind)


def _cdf_threshold(p: float) -> int:
    return int(math.floor(p * TWO32 + 0.5))


def const_delay_steps(d_ms: float, dt: float) -> int:
    """Constant delay: round-half-even(d / h) in fp64, at least one step."""
    return max(1, int(round(d_ms / dt)))


def quantised_normal_table(mean: float, sd: float, lo: float, dt: float):
    """Integer CDF table of step = max(1, round(max(d, lo) / dt)), d ~ N(mean, sd).

    Returns (s_min, thresholds) with step(w) = s_min + #{i : w >= thresholds[i]}.
    P(step <= s) = Phi(((s + 1/2) dt - mean) / sd) for s >= s_min: the clipped mass
    below lo lands on s_min.  The table stops at the first s whose threshold reaches
    2^32; a table that would exceed 255 steps is rejected (delays are stored in u8)."""
    s_min = max(1, int(round(lo / dt)))
    if s_min > MAX_DELAY_STEPS:        # the clipped mass below lo lands on s_min itself
        raise ValueError("delay distribution has mass above 255 steps")
    thr = []
    s = s_min
    while True:
        x = ((s + 0.5) * dt - mean) / sd
        phi = 0.5 * math.erfc(-x / math.sqrt(2.0))
        c = _cdf_threshold(phi)
        if c >= 4294967296:
            break
        thr.append(c)
        s += 1
        if s > MAX_DELAY_STEPS:
            raise ValueError("delay distribution has mass above 255 steps")
    return s_min, np.array(thr, dtype=np.uint64)


def delay_steps(dist, dt: float, w1, count: int):
    """Delay steps (uint8 values) for ``dist`` ('const' or 'normal_min')."""
    if dist.kind == "const":
        return np.full(count, const_delay_steps(dist.mean, dt), dtype=np.int64)
    if dist.kind == "normal_min":
        s_min, thr = quantised_normal_table(dist.mean, dist.sd, dist.lo, dt)
        w1 = np.asarray(w1, dtype=np.uint64)
        return s_min + np.searchsorted(thr, w1, side="right").astype(np.int64)
    raise ValueError(dist.kind)


def max_delay_steps(dist, dt: float) -> int:
    if dist.kind == "const":
        return const_delay_steps(dist.mean, dt)
    s_min, thr = quantised_normal_table(dist.mean, dist.sd, dist.lo, dt)
    return s_min + len(thr)


def poisson_table(rate_hz: float, dt: float):
    """Integer CDF table of Poisson(lambda), lambda = rate_hz * dt / 1000:
    count(w) = #{i : w >= thresholds[i]}."""
    lam = rate_hz * dt / 1000.0
    pmf = math.exp(-lam)
    cdf = pmf
    thr = []
    i = 0
    while True:
        c = _cdf_threshold(cdf)
        if c >= 4294967296 or i >= 255:
            break
        thr.append(c)
        i += 1
        pmf = pmf * lam / i
        cdf = cdf + pmf
    return np.array(thr, dtype=np.uint64)


MAX_GAP_TABLE = 1 << 22


def geometric_gap_table(p: float):
    """Integer CDF table of the gap G >= 0 between kept pairs when every pair is kept
    with probability p: P(G <= g) = 1 - (1 - p)^(g + 1), so G(w) = #{i : w >= thr[i]}.
    The power is accumulated by repeated multiplication in fp64, which rounds the same
    way in every IEEE implementation.  The table stops at the first threshold that
    reaches 2^32; p must be in (0, 1] and the table at most 2^22 entries long."""
    if not 0.0 < p <= 1.0:
        raise ValueError("p must be in (0, 1]")
    q = 1.0 - p
    qq = q
    thr = []
    while True:
        c = _cdf_threshold(1.0 - qq)
        if c >= 4294967296:
            break
        thr.append(c)
        if len(thr) > MAX_GAP_TABLE:
            raise ValueError("connection probability too small for the gap table")
        qq = qq * q
    return np.array(thr, dtype=np.uint64)


def inverse_table(thr, w):
    """#{i : w >= thr[i]} for a non-decreasing threshold table."""
    return np.searchsorted(np.asarray(thr, dtype=np.uint64), np.asarray(w, dtype=np.uint64),
                           side="right").astype(np.int64)
