"""Logical ranks on one GPU: per-rank layouts, image neurons and every communication
map against the oracle's per-rank construction, through the C ABI."""
import numpy as np
import pytest

from gpu_helpers import compare_maps, compare_rank, ensure_lib, gpu_build, oracle_layout
from oracle import connect as oc
from oracle import neuron as on
from paper_2512_09502_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_lib()


def _net(R, seed=3):
    return wl.balanced(240, 61, 30, 8, wl.DELAY_NORMAL, seed=seed, n_ranks=R)


@pytest.mark.parametrize("R", [2, 3, 7])
def test_rank_layouts_and_maps_match_oracle(R):
    net = _net(R)
    ctx = gpu_build(net)
    syn, ref = oracle_layout(net)
    for tau in range(R):
        compare_rank(ctx.get_connections(tau), ref["ranks"][tau])
    compare_maps(ctx, ref, R)
    assert ctx.stats()["n_images"] == sum(len(r["img_s"]) for r in ref["ranks"])
    ctx.destroy()


@pytest.mark.parametrize("exchange", ["p2p", "collective"])
def test_rank_simulation_matches_oracle(exchange):
    """Spikes routed through the maps reach the same targets: V after 100 steps
    within 1e-4 mV of the single-rank oracle, and the early spike trains equal."""
    R = 5
    net = _net(R, seed=11)
    net.drives = [wl.Drive(0, net.n_neurons, 16000.0, wl.J_E, 4)]
    ctx = gpu_build(net, exchange=exchange, spike_log_capacity=1 << 20, use_graph=False)
    syn, ref = oracle_layout(net, R=1)
    rk = ref["ranks"][0]
    sim = on.Simulator(net, rk["row_ptr"], rk["tgt"], rk["d"], rk["w"].astype(np.float32).astype(np.float64),
                       on.ring_slots_for(oc.max_delay(net)))
    spikes, _ = sim.run(100)
    ctx.simulate(100)
    V, _, _ = ctx.get_state(0, net.n_neurons)
    st, gid = ctx.get_spikes()
    o = sorted(spikes)
    g = sorted(zip(st.tolist(), gid.tolist()))
    assert len(o) > 0
    if o == g:
        assert np.max(np.abs(V - sim.V)) <= 1e-4
    else:
        # a threshold decision taken in different precisions may flip; everything
        # before the first flip must agree exactly
        first = next(k for k in range(min(len(o), len(g))) if o[k] != g[k]) if len(o) and len(g) else 0
        assert first > 0
    ctx.destroy()


def test_exchange_schemes_deliver_identical_events():
    R = 4
    net = _net(R, seed=12)
    net.drives = [wl.Drive(0, net.n_neurons, 16000.0, wl.J_E, 4)]
    a = gpu_build(net, exchange="p2p", use_graph=True)
    b = gpu_build(net, exchange="collective", use_graph=True)
    a.simulate(40)
    b.simulate(40)
    sa, sb = a.stats(), b.stats()
    assert sa["n_spikes"] == sb["n_spikes"] and sa["n_events"] == sb["n_events"]
    Va, _, _ = a.get_state(0, net.n_neurons)
    Vb, _, _ = b.get_state(0, net.n_neurons)
    assert np.max(np.abs(Va - Vb)) <= 1e-4


@pytest.mark.parametrize("R", [1, 3])
def test_pairwise_bernoulli(R):
    net = wl.tiny(wl.RULE_PAIRWISE_BERNOULLI, 0.1, n_src=300, n_tgt=200, n_ranks=R)
    ctx = gpu_build(net)
    _, ref = oracle_layout(net)
    for tau in range(R):
        compare_rank(ctx.get_connections(tau), ref["ranks"][tau])


@pytest.mark.parametrize("R,p,n_src,n_tgt", [(1, 0.1, 300, 200), (3, 0.1, 300, 200), (2, 1.0, 45, 33),
                                              (1, 0.0, 45, 33), (7, 0.013, 1000, 150), (1, 0.6, 77, 64)])
def test_pairwise_bernoulli_geometric(R, p, n_src, n_tgt):
    """Pairwise Bernoulli by geometric gaps: kept pairs, their order, delays and weights
    bit-exact against the oracle's walk on one and several ranks (maps included)."""
    net = wl.tiny(wl.RULE_PAIRWISE_BERNOULLI_GEOMETRIC, p, n_src=n_src, n_tgt=n_tgt, n_ranks=R)
    ctx = gpu_build(net)
    _, ref = oracle_layout(net)
    for tau in range(R):
        compare_rank(ctx.get_connections(tau), ref["ranks"][tau])
    for tau in range(R):
        for sig in range(R):
            if sig != tau:
                np.testing.assert_array_equal(ctx.get_maps(tau, sig, "R"), ref["ranks"][tau]["R"][sig])
                np.testing.assert_array_equal(ctx.get_maps(tau, sig, "S"), ref["S"][sig][tau])


def test_fixed_total_over_ranks():
    net = wl.tiny(wl.RULE_FIXED_TOTAL, 50_000, n_src=300, n_tgt=200, n_ranks=4)
    ctx = gpu_build(net)
    _, ref = oracle_layout(net)
    for tau in range(4):
        compare_rank(ctx.get_connections(tau), ref["ranks"][tau])


def test_multi_area_over_ranks():
    """Multi-area stand-in over logical ranks: fixed-total and fixed in-degree blocks
    of every projection x rank, image maps, bit-exact per rank."""
    net = wl.multi_area(seed=1234, n_areas=6, area_mean=300.0, n_ranks=8)
    ctx = gpu_build(net)
    _, ref = oracle_layout(net)
    for tau in range(8):
        compare_rank(ctx.get_connections(tau), ref["ranks"][tau])
        for sig in range(8):
            if sig != tau:
                np.testing.assert_array_equal(ctx.get_maps(tau, sig, "R"), ref["ranks"][tau]["R"][sig])
                np.testing.assert_array_equal(ctx.get_maps(tau, sig, "S"), ref["S"][sig][tau])


def _every_rule_net(R):
    """One projection of every rule, including one-to-one and all-to-all, on four
    populations of uneven sizes."""
    pops = [wl.Population(n) for n in (211, 211, 57, 90)]
    w, d = wl.Dist(wl.W_NORMAL_SIGN, 40.0, 8.0), wl.DELAY_NORMAL
    P = wl.Projection
    projs = [P(0, 211, 211, 211, wl.Rule(wl.RULE_ONE_TO_ONE, 0), w, d, 3),
             P(422, 57, 479, 90, wl.Rule(wl.RULE_ALL_TO_ALL, 0), w, d, 4),
             P(0, 211, 422, 57, wl.Rule(wl.RULE_FIXED_INDEGREE, 5), w, d, 5),
             P(211, 211, 0, 211, wl.Rule(wl.RULE_FIXED_TOTAL, 900), w, d, 6),
             P(479, 90, 211, 211, wl.Rule(wl.RULE_PAIRWISE_BERNOULLI, 0.05), w, d, 7),
             P(211, 211, 479, 90, wl.Rule(wl.RULE_ALL_TO_ALL, 0), w, d, 8)]
    return wl.Network("every_rule", pops, projs, n_ranks=R)


@pytest.mark.parametrize("R,xi", [(1, 0.0), (4, 0.0), (5, 1.0)])
def test_one_to_one_and_all_to_all(R, xi):
    """One-to-one and all-to-all beside the other rules: layouts bit-exact and every map
    equal to the oracle's on one and several ranks (xi applies to the random rules only)."""
    net = _every_rule_net(R)
    ctx = gpu_build(net, xi=xi)
    _, ref = oracle_layout(net, xi=xi)
    for tau in range(R):
        compare_rank(ctx.get_connections(tau), ref["ranks"][tau])
    if R > 1:
        compare_maps(ctx, ref, R)
    n_pb = sum(int(np.sum(r["src"] >= 479)) for r in ref["ranks"])       # the Bernoulli block's sources
    assert ctx.stats()["n_synapses"] == 211 + 57 * 90 + 5 * 57 + 900 + n_pb + 211 * 90
    ctx.destroy()


def test_one_to_one_and_all_to_all_dry_run():
    """Uncounted rules only (fixed in-degree, one-to-one, all-to-all): a dry run of rank 2
    of 4 builds that rank's rows and R/L maps of the full build."""
    pops = [wl.Population(n) for n in (300, 300, 40)]
    w, d = wl.Dist(wl.W_NORMAL_SIGN, 40.0, 8.0), wl.DELAY_NORMAL
    P = wl.Projection
    net = wl.Network("uncounted", pops, [P(0, 300, 300, 300, wl.Rule(wl.RULE_ONE_TO_ONE, 0), w, d, 3),
                                         P(600, 40, 0, 300, wl.Rule(wl.RULE_ALL_TO_ALL, 0), w, d, 4),
                                         P(300, 300, 0, 300, wl.Rule(wl.RULE_FIXED_INDEGREE, 7), w, d, 5)],
                     n_ranks=4)
    dry = gpu_build(net, dry_run_rank=2)
    _, ref = oracle_layout(net)
    compare_rank(dry.get_connections(2), ref["ranks"][2])
    for sig in (0, 1, 3):
        np.testing.assert_array_equal(dry.get_maps(2, sig, "R"), ref["ranks"][2]["R"][sig])
        np.testing.assert_array_equal(dry.get_maps(2, sig, "L"), ref["ranks"][2]["L"][sig])
