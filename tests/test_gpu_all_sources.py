"""All-sources images (Methods, "Remote connections", threshold xi): projections whose
expected connections per source reach xi give every source an image on every rank
holding their targets.  Layouts and every map against the oracle's per-rank
construction with the same threshold, through the C ABI; the dynamics do not depend on
xi."""
import numpy as np
import pytest

from gpu_helpers import compare_maps, compare_rank, ensure_lib, gpu_build, oracle_layout
from paper_2512_09502_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_lib()


@pytest.mark.parametrize("R,xi", [(2, 1.0), (3, 1.0), (8, 1.0), (5, 0.5), (4, 0.0)])
def test_all_sources_layouts_and_maps_match_oracle(R, xi):
    net = wl.mixed_rules(n_ranks=R)
    ctx = gpu_build(net, xi=xi)
    _, ref = oracle_layout(net, xi=xi)
    for tau in range(R):
        compare_rank(ctx.get_connections(tau), ref["ranks"][tau])
    compare_maps(ctx, ref, R)
    assert ctx.stats()["n_images"] == sum(len(r["img_s"]) for r in ref["ranks"])
    ctx.destroy()


def test_all_sources_images_only_on_ranks_with_targets():
    """RemoteConnect from the 125 neurons of rank 5 onto the 125 of rank 3 (8 ranks) with
    K = 1, i.e. 1 connection per source: at xi = 1 rank 3 holds an image of each source
    and no other rank holds any; at xi = 1.5 only of the sources it uses."""
    pops = [wl.Population(1000), wl.Population(1000)]
    pr = wl.Projection(5, 125, 1003, 125, wl.Rule(wl.RULE_FIXED_INDEGREE, 1), wl.Dist(wl.W_CONST, 1.0),
                       wl.Dist(wl.D_CONST, 1.0), 9, src_stride=8, tgt_stride=8)
    net = wl.Network("k1_rank5_to_rank3", pops, [pr], n_ranks=8)
    for xi in (1.0, 1.5):
        ctx = gpu_build(net, xi=xi)
        _, ref = oracle_layout(net, xi=xi)
        n_img = []
        for tau in range(8):
            c = ctx.get_connections(tau)
            compare_rank(c, ref["ranks"][tau])
            n_img.append(len(c["row_ptr"]) - 1 - ref["ranks"][tau]["M"])
        compare_maps(ctx, ref, 8)
        if xi == 1.0:
            assert n_img == [0, 0, 0, 125, 0, 0, 0, 0]
        else:
            assert 0 < n_img[3] < 125 and sum(n_img) == n_img[3]


@pytest.mark.parametrize("exchange", ["p2p", "collective"])
def test_all_sources_images_leave_the_dynamics_unchanged(exchange):
    """Images without connections route spikes to empty rows: the same spikes and
    events as with flagged images only."""
    R = 6
    net = wl.mixed_rules(n_ranks=R)
    a = gpu_build(net, exchange=exchange, use_graph=True)
    b = gpu_build(net, exchange=exchange, use_graph=True, xi=1.0)
    assert b.stats()["n_images"] > a.stats()["n_images"]
    a.simulate(200)
    b.simulate(200)
    sa, sb = a.stats(), b.stats()
    assert sa["n_spikes"] > 0
    assert sa["n_spikes"] == sb["n_spikes"] and sa["n_events"] == sb["n_events"]
    Va, _, _ = a.get_state(0, net.n_neurons)
    Vb, _, _ = b.get_state(0, net.n_neurons)
    assert np.max(np.abs(Va - Vb)) <= 1e-4


@pytest.mark.parametrize("r", [0, 4])
def test_all_sources_dry_run(r):
    """A dry run with the threshold builds the rank's rows and R/L maps of the full
    build.  K_E = 4 over 60 targets per rank and 240 sources is exactly 1 connection per
    source (forced at xi = 1), K_I = 1 over 61 sources is not."""
    R = 5
    net = wl.balanced(240, 61, 4, 1, wl.DELAY_NORMAL, seed=3, n_ranks=R)
    full = gpu_build(net, xi=1.0)
    dry = gpu_build(net, xi=1.0, dry_run_rank=r)
    _, ref = oracle_layout(net, xi=1.0)
    compare_rank(dry.get_connections(r), ref["ranks"][r])
    for sig in range(R):
        if sig != r:
            for which in ("R", "L"):
                np.testing.assert_array_equal(dry.get_maps(r, sig, which), full.get_maps(r, sig, which))
                np.testing.assert_array_equal(dry.get_maps(r, sig, which), ref["ranks"][r][which][sig])
