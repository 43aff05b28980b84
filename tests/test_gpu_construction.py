"""GPU parity of network construction against the oracle, through the C ABI:
(source, target, delay) records bit-exact, weights within 4 fp32 ulp."""
import numpy as np
import pytest

from gpu_helpers import compare_rank, ensure_lib, f32_ulp_distance, gpu_build, oracle_layout
from oracle import connect as oc
from paper_2512_09502_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_lib()


def _check(net, fmt="f32"):
    ctx = gpu_build(net, weight_format=fmt)
    syn, ref = oracle_layout(net)
    got = ctx.get_connections(0)
    compare_rank(got, ref["ranks"][0], fmt)
    st = ctx.stats()
    assert st["n_synapses"] == len(syn["src"])
    ctx.destroy()


def test_balanced_5k_bit_exact():
    _check(wl.balanced_small())


@pytest.mark.parametrize("rb", [8, 9, 10])
@pytest.mark.parametrize("items", [8, 12, 16])
@pytest.mark.parametrize("n,R,key_bits,passes", [(16001, 1, 20, {8: 3, 9: 3, 10: 2}),
                                                 (2001, 1, 17, {8: 3, 9: 2, 10: 2}),
                                                 (48001, 3, 22, {8: 3, 9: 3, 10: 3})])
def test_every_sort_kernel_width(rb, items, n, R, key_bits, passes):
    """Every digit width and tile (8, 12, 16 records per thread) of the radix sort on
    (rank slot, source, delay) keys: 14 source + 6 delay bits (digits 8, 8, 4, or 10, 10
    when the widest is 10), 11 + 6 bits (8, 8, 1, or 8, 9), and on 3 ranks 2 slot + 14
    source + 6 delay bits (8, 8, 6), over several tiles with ragged tails, bit-exact
    against the oracle."""
    net = wl.balanced(n * 4 // 5, n - n * 4 // 5, 30, 8, wl.DELAY_NORMAL, seed=rb * 100 + items, n_ranks=R)
    ctx = gpu_build(net, radix_bits=rb, sort_items=items)
    syn, ref = oracle_layout(net)
    for tau in range(R):
        compare_rank(ctx.get_connections(tau), ref["ranks"][tau])
    st = ctx.stats()
    assert st["n_synapses"] == len(syn["src"]) and st["radix_bits"] == rb
    assert st["key_bits"] == key_bits and st["sort_passes"] == passes[rb]
    ctx.destroy()


@pytest.mark.parametrize("ne,ni,ke,ki", [(300, 75, 40, 10), (1001, 250, 37, 9), (4097, 3, 5, 1), (17, 2, 1, 1)])
def test_ragged_sizes_normal_delays(ne, ni, ke, ki):
    _check(wl.balanced(ne, ni, ke, ki, wl.DELAY_NORMAL, seed=ne))


def test_indegree_beyond_source_count():
    """In-degree scaling (the paper's appendix on in-degree): K = 10x the neurons' count
    of its population, so every target draws each source ~10 times (multapses)."""
    net = wl.indegree_scaling(10, neurons_at_1=1000)
    assert net.projections[0].rule.param == 90000 and net.populations[0].n == 80
    _check(net)


def test_delay_tables_match_oracle():
    from oracle import sampling as sm
    net = wl.balanced(300, 75, 40, 10, wl.DELAY_NORMAL)
    ctx = gpu_build(net)
    smin, thr = ctx.get_delay_table(0)
    o_smin, o_thr = sm.quantised_normal_table(1.5, 0.75, 0.1, 0.1)
    assert smin == o_smin
    np.testing.assert_array_equal(thr.astype(np.uint64), o_thr)


def test_single_neuron_autapses_and_extreme_delays():
    p = wl.BALANCED_PARAMS
    net = wl.Network("one", [wl.Population(1, p)],
                     [wl.Projection(0, 1, 0, 1, wl.Rule(wl.RULE_FIXED_INDEGREE, 3),
                                    wl.Dist(wl.W_CONST, 5.0), wl.Dist(wl.D_CONST, 0.01), 1),
                      wl.Projection(0, 1, 0, 1, wl.Rule(wl.RULE_FIXED_INDEGREE, 2),
                                    wl.Dist(wl.W_NORMAL_SIGN, -3.0, 1.0), wl.Dist(wl.D_CONST, 25.4), 2)])
    _check(net)


def test_sources_without_connections_have_empty_rows():
    p = wl.BALANCED_PARAMS
    net = wl.Network("gap", [wl.Population(50, p), wl.Population(5000, p)],
                     [wl.Projection(20, 10, 50, 5000, wl.Rule(wl.RULE_FIXED_INDEGREE, 7),
                                    wl.Dist(wl.W_NORMAL_SIGN, 10.0, 2.0), wl.DELAY_NORMAL, 9)])
    _check(net)


def test_fixed_total_one_rank():
    net = wl.tiny(wl.RULE_FIXED_TOTAL, 60_000, n_src=300, n_tgt=200)
    _check(net)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_low_precision_weight_formats(fmt):
    _check(wl.balanced(1001, 250, 37, 9, wl.DELAY_NORMAL, seed=3), fmt)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_low_precision_weight_formats_over_ranks(fmt):
    """BF16 and FP16 (power-of-two scale per source) weights on four logical ranks: every
    rank's layout bit-exact and its weights within the format's rounding of the oracle's,
    image rows included (their scale is their source's)."""
    net = wl.balanced(1001, 250, 37, 9, wl.DELAY_NORMAL, seed=4, n_ranks=4)
    ctx = gpu_build(net, weight_format=fmt)
    _, ref = oracle_layout(net)
    for tau in range(4):
        compare_rank(ctx.get_connections(tau), ref["ranks"][tau], fmt)
    ctx.destroy()


def test_full_size_sampled_parity():
    """The scaled balanced network at full size (5.625G synapses): exact totals, exact
    row sums, and sampled targets regenerated by the oracle found in their source
    rows with identical delay and weight."""
    net = wl.balanced_scaled(1.0)
    ctx = gpu_build(net)
    st = ctx.stats()
    assert st["n_synapses"] == net.n_synapses_fixed() == 5_625_000_000
    rng = np.random.default_rng(0)
    for t in rng.integers(0, net.n_neurons, size=3):
        for pid in (0, 1):
            one = oc.fixed_indegree_target(net, pid, int(t))
            for s in np.unique(one["src"])[:25]:
                tgt, w, d = ctx.get_row(0, int(s))
                assert np.all(np.diff(d.astype(np.int64)) >= 0)          # delay-ordered row
                m = tgt == t
                mine = np.nonzero(one["src"] == s)[0]
                order = mine[np.argsort(one["d"][mine], kind="stable")]    # (delay, k) order
                np.testing.assert_array_equal(d[m].astype(np.int64), one["d"][order])
                assert f32_ulp_distance(w[m], one["w"][order].astype(np.float32)).max() <= 4
    ctx.destroy()


def test_multi_area_batched_blocks():
    """Multi-area stand-in (8 areas, 64 fixed-total intra blocks per area plus
    fixed in-degree inter-area blocks, uneven sizes) built in one generation launch."""
    net = wl.multi_area(seed=1234, n_areas=8, area_mean=400.0)
    assert len(net.projections) > 8 * 64
    _check(net)


def _runs(row_ptr, key):
    """Starts of the maximal runs of equal `key` inside every row (row starts included)."""
    starts = set(int(x) for x in row_ptr[:-1] if x < row_ptr[-1])
    starts.update(int(i) for i in np.nonzero(key[1:] != key[:-1])[0] + 1)
    return np.array(sorted(starts), dtype=np.int64)


@pytest.mark.parametrize("R", [1, 3])
def test_delay_runs_recovered_from_row_starts_and_delays(R):
    """The layout stores no per-(source, delay) run offsets: every row is non-decreasing in
    its delays, so its runs are its maximal stretches of equal delay.  The run starts
    recovered that way from the device's row starts and delay array equal the (source,
    delay) run starts of the oracle's layout, on one rank and on three."""
    net = wl.balanced(1200, 300, 60, 15, wl.DELAY_NORMAL, seed=17, n_ranks=R)
    ctx = gpu_build(net)
    _, ref = oracle_layout(net)
    for tau in range(R):
        got = ctx.get_connections(tau)
        rp, d = got["row_ptr"], got["d"].astype(np.int64)
        for r in range(len(rp) - 1):
            assert np.all(np.diff(d[rp[r]:rp[r + 1]]) >= 0), (tau, r)
        row_of = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        gpu_runs = _runs(rp, row_of * 1024 + d)
        rk = ref["ranks"][tau]
        oracle_runs = _runs(rk["row_ptr"], rk["src"].astype(np.int64) * 1024 + rk["d"])
        np.testing.assert_array_equal(gpu_runs, oracle_runs)
    ctx.destroy()
