"""Pins of the oracle's connection rules (no GPU)."""
import numpy as np
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
