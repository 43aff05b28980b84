"""Pins of the oracle's connection rules (no GPU)."""
import numpy as np
import pytest
from scipy import stats

from oracle import connect as oc
from oracle import layout as ol
from paper_2512_09502_gb300 import workloads as wl


def test_fixed_indegree_exact_indegree():
    net = wl.balanced_small()
    syn = oc.generate(net)
    assert len(syn["src"]) == 2_500_000 == net.n_synapses_fixed()
    indeg = np.bincount(syn["tgt"], minlength=5000)
    assert np.all(indeg == 500)
    e = syn["src"] < 4000
    assert np.all(np.bincount(syn["tgt"][e], minlength=5000) == 400)
    assert np.all(np.bincount(syn["tgt"][~e], minlength=5000) == 100)
    assert np.all(syn["d"] == 15)
    assert np.all(syn["w"][e] > 0) and np.all(syn["w"][~e] < 0)
    assert np.all(np.diff(syn["gidx"]) == 1)


def test_fixed_indegree_sources_uniform():
    net = wl.tiny(wl.RULE_FIXED_INDEGREE, 5000, n_src=10, n_tgt=20)
    syn = oc.generate(net)
    cnt = np.bincount(syn["src"], minlength=10)
    assert stats.chisquare(cnt).pvalue > 1e-3
    assert syn["src"].min() >= 0 and syn["src"].max() < 10
    assert syn["tgt"].min() >= 10 and syn["tgt"].max() < 30


def test_fixed_total_exact_and_uniform_cells():
    net = wl.tiny(wl.RULE_FIXED_TOTAL, 60_000, n_src=10, n_tgt=12)
    syn = oc.generate(net)
    assert len(syn["src"]) == 60_000
    cells = np.bincount((syn["src"]) * 12 + (syn["tgt"] - 10), minlength=120)
    assert stats.chisquare(cells).pvalue > 1e-3


def test_pairwise_bernoulli_limits_and_count():
    full = oc.generate(wl.tiny(wl.RULE_PAIRWISE_BERNOULLI, 1.0))
    pairs = set(zip(full["src"].tolist(), full["tgt"].tolist()))
    assert len(full["src"]) == 400 and len(pairs) == 400         # every pair once
    none = oc.generate(wl.tiny(wl.RULE_PAIRWISE_BERNOULLI, 0.0))
    assert len(none["src"]) == 0
    n = 300 * 200
    net = wl.tiny(wl.RULE_PAIRWISE_BERNOULLI, 0.1, n_src=300, n_tgt=200)
    syn = oc.generate(net)
    assert abs(len(syn["src"]) - 0.1 * n) < 5 * np.sqrt(n * 0.1 * 0.9)
    assert len(set(zip(syn["src"].tolist(), syn["tgt"].tolist()))) == len(syn["src"])  # no multapses
    col = np.bincount(syn["src"], minlength=300)
    assert stats.chisquare(col).pvalue > 1e-4


def test_per_target_generation_equals_full():
    net = wl.balanced_small()
    syn = oc.generate(net)
    for t in [0, 17, 4999]:
        one = oc.fixed_indegree_target(net, 0, t)
        m = (syn["tgt"] == t) & (syn["proj"] == 0)
        np.testing.assert_array_equal(one["src"], syn["src"][m])
        np.testing.assert_array_equal(one["d"], syn["d"][m])
        np.testing.assert_array_equal(one["w"], syn["w"][m])


def test_partition_invariance_and_layout_order():
    """Every partition flattens to the 1-rank multiset; rows hold (source, delay)
    sorted connections, ties in generation order."""
    net = wl.balanced(300, 75, 40, 10, wl.DELAY_NORMAL, seed=5)
    syn = oc.generate(net)
    ref = ol.flatten(ol.build_all(syn, ol.round_robin(net.n_neurons, 1))["ranks"],
                     ol.round_robin(net.n_neurons, 1))
    ref = ref[np.lexsort(ref.T[::-1])]
    for R in [2, 3, 7]:
        part = ol.round_robin(net.n_neurons, R)
        out = ol.build_all(syn, part)
        flat = ol.flatten(out["ranks"], part)
        flat = flat[np.lexsort(flat.T[::-1])]
        np.testing.assert_array_equal(flat, ref)
        for rk in out["ranks"]:
            rp = rk["row_ptr"]
            assert rp[-1] == len(rk["tgt"])
            for r in range(len(rp) - 1):
                a, b = rp[r], rp[r + 1]
                key = rk["d"][a:b] * (1 << 40) + rk["gidx"][a:b]
                assert np.all(np.diff(key) > 0)
                assert np.all(rk["src"][a:b] == rk["src"][a])


def _geom_net(n_src, n_tgt, p, seed=5):
    pr = wl.Projection(0, n_src, n_src, n_tgt, wl.Rule(wl.RULE_PAIRWISE_BERNOULLI_GEOMETRIC, p),
                       wl.Dist(wl.W_CONST, 1.0, 0.0), wl.Dist(wl.D_CONST, 1.0), seed)
    return wl.Network("geom", [wl.Population(n_src), wl.Population(n_tgt)], [pr], [])


def test_geometric_gap_table_against_scipy():
    """thr_g = round(P(G <= g) 2^32) for the number of failures before a success:
    scipy's geom counts trials, so P(G <= g) = geom.cdf(g + 1)."""
    from oracle import sampling as sm
    for p in (0.5, 0.1, 0.013, 0.001):
        thr = sm.geometric_gap_table(p)
        g = np.arange(len(thr))
        ref = np.floor(stats.geom.cdf(g + 1, p) * 2.0 ** 32 + 0.5)
        assert np.abs(thr.astype(np.float64) - ref).max() <= 1.0
        assert stats.geom.cdf(len(thr) + 1, p) * 2.0 ** 32 + 0.5 >= 2.0 ** 32 - 1   # stops at the top
    assert len(sm.geometric_gap_table(1.0)) == 0           # p = 1: every gap is 0


def test_geometric_bernoulli_limits_and_pair_independence():
    """p = 1 keeps every pair; per-target counts follow Binomial(n_src, p); every source
    is equally likely; gaps between kept sources are geometric; no multapses."""
    all_pairs = oc.generate(_geom_net(13, 7, 1.0))
    assert len(all_pairs["c"]) == 13 * 7
    np.testing.assert_array_equal(all_pairs["c"], np.arange(13 * 7))
    assert len(oc.generate(_geom_net(13, 7, 0.0))["c"]) == 0
    n_src, n_tgt, p = 200, 400, 0.1
    syn = oc.generate(_geom_net(n_src, n_tgt, p))
    s = syn["src"]
    t = syn["tgt"] - n_src
    assert (np.diff(syn["c"]) > 0).all()                   # (target, source) order, no multapses
    counts = np.bincount(t, minlength=n_tgt)
    assert abs(counts.mean() - n_src * p) < 4 * np.sqrt(n_src * p * (1 - p) / n_tgt)
    assert abs(counts.var() / (n_src * p * (1 - p)) - 1.0) < 0.25
    src_hist = np.bincount(s, minlength=n_src)             # inclusion per source ~ Binomial(n_tgt, p)
    chi2 = ((src_hist - n_tgt * p) ** 2 / (n_tgt * p)).sum()
    assert stats.chi2.sf(chi2, n_src - 1) > 1e-3
    gaps = []                                              # gaps between kept sources of a target
    for k in range(n_tgt):
        ss = np.sort(s[t == k])
        gaps += list(np.diff(ss) - 1)
    gaps = np.array(gaps)
    kmax = 30
    obs = np.array([np.count_nonzero(gaps == k) for k in range(kmax)] + [np.count_nonzero(gaps >= kmax)])
    pmf = np.array([stats.geom.pmf(k + 1, p) for k in range(kmax)] + [stats.geom.sf(kmax, p)])
    exp = pmf / pmf.sum() * len(gaps)
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert stats.chi2.sf(chi2, kmax) > 1e-3


def test_geometric_and_pairwise_bernoulli_totals_agree():
    """Both realizations of pairwise Bernoulli keep Binomial(n_src n_tgt, p) pairs."""
    n_src, n_tgt, p = 300, 300, 0.05
    tot_g = len(oc.generate(_geom_net(n_src, n_tgt, p, seed=9))["c"])
    net_pb = _geom_net(n_src, n_tgt, p, seed=9)
    net_pb.projections[0] = wl.Projection(0, n_src, n_src, n_tgt, wl.Rule(wl.RULE_PAIRWISE_BERNOULLI, p),
                                          wl.Dist(wl.W_CONST, 1.0, 0.0), wl.Dist(wl.D_CONST, 1.0), 9)
    tot_p = len(oc.generate(net_pb)["c"])
    sd = np.sqrt(n_src * n_tgt * p * (1 - p))
    for tot in (tot_g, tot_p):
        assert abs(tot - n_src * n_tgt * p) < 4 * sd


def test_all_to_all_is_pairwise_bernoulli_at_p1():
    """All-to-all makes every (target, source) pair once, in (target, source) order, with
    the synapse counter i_t n_src + i_s: exactly the pairs, delays and weights of the
    pairwise Bernoulli rule at p = 1, whose pairs come through its own test stream."""
    pops = [wl.Population(37), wl.Population(23)]
    w, d = wl.Dist(wl.W_NORMAL_SIGN, 40.0, 8.0), wl.DELAY_NORMAL
    a2a = wl.Network("a2a", pops, [wl.Projection(0, 37, 37, 23, wl.Rule(wl.RULE_ALL_TO_ALL, 0), w, d, 9)])
    pb1 = wl.Network("pb1", pops, [wl.Projection(0, 37, 37, 23, wl.Rule(wl.RULE_PAIRWISE_BERNOULLI, 1.0), w, d, 9)])
    x, y = oc.generate(a2a), oc.generate(pb1)
    assert len(x["src"]) == 37 * 23
    for k in ("src", "tgt", "d", "w", "c"):
        np.testing.assert_array_equal(x[k], y[k])
    pairs = set(zip(x["src"].tolist(), x["tgt"].tolist()))
    assert pairs == {(s, 37 + t) for s in range(37) for t in range(23)}
    assert a2a.n_synapses_fixed() == 37 * 23


def test_one_to_one_pairs_and_draws():
    """One-to-one connects target i from source i, once each.  Its counter is the target
    index, so its delays and weights are those of fixed in-degree K = 1 from a single
    source neuron (counter i_t K + k = i_t), generated by the other rule's code."""
    n = 150
    pops = [wl.Population(n), wl.Population(n), wl.Population(1)]
    w, d = wl.Dist(wl.W_NORMAL_SIGN, -30.0, 6.0), wl.DELAY_NORMAL
    one = wl.Network("o2o", pops, [wl.Projection(0, n, n, n, wl.Rule(wl.RULE_ONE_TO_ONE, 0), w, d, 4)])
    fi1 = wl.Network("fi1", pops, [wl.Projection(2 * n, 1, n, n, wl.Rule(wl.RULE_FIXED_INDEGREE, 1), w, d, 4)])
    x, y = oc.generate(one), oc.generate(fi1)
    np.testing.assert_array_equal(x["src"], np.arange(n))
    np.testing.assert_array_equal(x["tgt"], n + np.arange(n))
    np.testing.assert_array_equal(y["src"], np.full(n, 2 * n))
    for k in ("tgt", "d", "w", "c"):
        np.testing.assert_array_equal(x[k], y[k])
    bad = wl.Network("bad", pops, [wl.Projection(0, n, n, n - 1, wl.Rule(wl.RULE_ONE_TO_ONE, 0), w, d, 4)])
    with pytest.raises(ValueError):
        oc.generate(bad)
