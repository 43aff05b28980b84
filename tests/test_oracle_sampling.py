"""Pins of the oracle's variates and integer CDF tables (no GPU)."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import philox as ph
from oracle import sampling as sm


def test_uniform_index_boundaries():
    """floor(w n / 2^32) steps from k-1 to k exactly at w = ceil(k 2^32 / n)."""
    for n in [1, 3, 10, 4000, 500_000, 2**31 + 7]:
        for k in [1, n // 2, n - 1]:
            if k <= 0:
                continue
            w = -(-(k << 32) // n)
            assert int(sm.uniform_index(np.uint64(w), n)) == k
            assert int(sm.uniform_index(np.uint64(w - 1), n)) == k - 1
        assert int(sm.uniform_index(np.uint64(0xFFFFFFFF), n)) == n - 1


def test_uniform_index_chi_square():
    b = ph.stream(np.arange(200_000, dtype=np.uint64), 0, 0, 1234)
    idx = sm.uniform_index(b[0], 10).astype(np.int64)
    cnt = np.bincount(idx, minlength=10)
    assert stats.chisquare(cnt).pvalue > 1e-3


def test_u01_exact_and_open():
    w = np.array([0, 511, 512, 0xFFFFFFFF], dtype=np.uint64)
    u = sm.u01(w)
    assert u[0] == 0.5 * 2**-23 and u[1] == u[0]
    assert u[2] == 1.5 * 2**-23
    assert u[3] == 1.0 - 0.5 * 2**-23
    assert np.all(u.astype(np.float32).astype(np.float64) == u)   # exact in fp32


def test_box_muller_special_cases():
    """u1 ~ 1/2 gives |z| ~ sqrt(2 ln 2); u2 ~ 0 gives cos ~ +1, u2 ~ 1/2 gives -1,
    u2 ~ 1/4 gives ~0."""
    half = np.array([1 << 31], dtype=np.uint64)                 # u = 1/2 + 2^-24
    r = math.sqrt(2 * math.log(2))
    assert abs(sm.box_muller(half, np.array([0], np.uint64))[0] - r) < 1e-6
    assert abs(sm.box_muller(half, half)[0] + r) < 1e-6
    assert abs(sm.box_muller(half, np.array([1 << 30], np.uint64))[0]) < 1e-6
    tiny = np.array([0], dtype=np.uint64)                       # u1 = 2^-24: the largest |z|
    assert abs(sm.box_muller(tiny, np.array([0], np.uint64))[0] - math.sqrt(48 * math.log(2))) < 1e-6


def test_box_muller_is_standard_normal():
    b = ph.stream(np.arange(100_000, dtype=np.uint64), 0, 0, 42)
    z = sm.box_muller(b[2], b[3])
    assert abs(z.mean()) < 4 / math.sqrt(len(z))
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / len(z))
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_normal_weights_keep_sign():
    from paper_2512_09502_gb300.workloads import Dist
    b = ph.stream(np.arange(10000, dtype=np.uint64), 0, 0, 3)
    w = sm.weight_values(Dist("normal_sign", 1.0, 2.0), b[2], b[3], 10000)
    assert w.min() == 0.0 and (w == 0).sum() > 1000      # clamped, not redrawn
    w = sm.weight_values(Dist("normal_sign", -1.0, 2.0), b[2], b[3], 10000)
    assert w.max() == 0.0
    w = sm.weight_values(Dist("normal_sign", 87.8, 8.78), b[2], b[3], 10000)
    assert abs(w.mean() - 87.8) < 4 * 8.78 / 100 and abs(w.std() - 8.78) < 0.2


def test_const_delay_rounding():
    assert sm.const_delay_steps(1.5, 0.1) == 15       # 1.5/0.1 = 15.000000000000002
    assert sm.const_delay_steps(0.04, 0.1) == 1      # at least one step
    assert sm.const_delay_steps(0.25, 0.1) == 2      # half-even: 2.5 -> 2


def test_quantised_normal_table_probabilities():
    """Table thresholds equal floor(P(step <= s) 2^32 + 1/2) with P from scipy's
    normal CDF (an independent implementation), and the tail stops below 2^-32."""
    mean, sd, lo, dt = 1.5, 0.75, 0.1, 0.1
    s_min, thr = sm.quantised_normal_table(mean, sd, lo, dt)
    assert s_min == 1
    s = s_min + np.arange(len(thr))
    p = stats.norm.cdf(((s + 0.5) * dt - mean) / sd)
    assert np.max(np.abs(thr.astype(np.float64) - p * 2**32)) <= 1.0
    assert np.all(np.diff(thr.astype(np.int64)) >= 0)
    # the next step's CDF rounds to 2^32
    p_next = stats.norm.cdf(((s[-1] + 1.5) * dt - mean) / sd)
    assert p_next * 2**32 + 0.5 >= 2**32 - 1
    # clipped mass below lo lands on s_min
    assert abs(thr[0] / 2**32 - stats.norm.cdf((1.5 * dt - mean) / sd)) < 1e-9


def test_quantised_normal_sample_chi_square():
    from paper_2512_09502_gb300.workloads import Dist
    dist = Dist("normal_min", 1.5, 0.75, 0.1)
    b = ph.stream(np.arange(400_000, dtype=np.uint64), 0, 0, 11)
    d = sm.delay_steps(dist, 0.1, b[1], 400_000)
    assert d.min() >= 1
    s_min, thr = sm.quantised_normal_table(1.5, 0.75, 0.1, 0.1)
    edges = np.arange(s_min, s_min + len(thr) + 1)
    cdf = stats.norm.cdf(((edges + 0.5) * 0.1 - 1.5) / 0.75)
    pk = np.diff(np.concatenate([[0.0], cdf[:-1], [1.0]]))
    cnt = np.bincount(d - s_min, minlength=len(pk))[:len(pk)]
    keep = pk * len(d) > 20
    obs = np.append(cnt[keep], cnt[~keep].sum())
    exp = np.append(pk[keep], pk[~keep].sum()) * len(d)
    assert stats.chisquare(obs, exp).pvalue > 1e-3


def test_delay_table_rejects_above_255():
    with pytest.raises(ValueError):
        sm.quantised_normal_table(25.0, 2.0, 0.1, 0.1)
    # clipped below at 30 ms = 300 steps with the normal's mass far below it: every
    # delay would be the clip step itself, which does not fit a u8
    with pytest.raises(ValueError):
        sm.quantised_normal_table(1.5, 0.75, 30.0, 0.1)


def test_delay_table_clip_step_at_255_is_kept():
    """lo = 25.5 ms at dt = 0.1 ms: the clip step is 255, the largest u8 delay, and all
    the normal's mass lies below it, so the table is empty and every delay is 255."""
    s_min, thr = sm.quantised_normal_table(1.5, 0.75, 25.5, 0.1)
    assert s_min == 255 and len(thr) == 0
    assert sm.max_delay_steps(wl_dist_normal(1.5, 0.75, 25.5), 0.1) == 255


def wl_dist_normal(mean, sd, lo):
    from paper_2512_09502_gb300 import workloads as wl
    return wl.Dist(wl.D_NORMAL_MIN, mean, sd, lo)


def test_poisson_table_matches_scipy():
    thr = sm.poisson_table(8000.0, 0.1)
    k = np.arange(len(thr))
    p = stats.poisson.cdf(k, 0.8)
    assert np.max(np.abs(thr.astype(np.float64) - p * 2**32)) <= 1.0
    b = ph.stream(np.arange(300_000, dtype=np.uint64), 0, 3, 5)
    cnt = sm.inverse_table(thr, b[0])
    assert abs(cnt.mean() - 0.8) < 4 * math.sqrt(0.8 / len(cnt))
    assert abs(cnt.var() - 0.8) < 0.02
