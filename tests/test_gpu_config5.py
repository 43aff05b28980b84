"""The multi-area network over 128 logical ranks (round robin), on one GPU, through the
C ABI (paper, Methods, "Remote connections" and both subsections on creating the remote
connection structures, for point-to-point and for collective communication).

At a reduced size (4 areas of about 750 neurons, 3,012 neurons, 0.6M synapses) the
128-rank build reaches what small rank counts do not: a routing fan-out of up to 127
image ranks per source, about 24 local neurons per rank beside ~1,800 image rows, a
rank slot of 7 bits in the sort key and 261 projections in 30,000+ (projection, rank)
blocks.  Every rank's layout and every R/L/S/T/P/H/I/G/Q map must equal the oracle's
per-rank construction bit for bit.  Then 1,000 graph-captured steps route spikes
through the maps under both exchange schemes."""
import dataclasses

import numpy as np
import pytest

from gpu_helpers import compare_maps, compare_rank, ensure_lib, gpu_build, oracle_layout
from oracle import connect as oc
from oracle import layout as ol
from oracle import neuron as on
from paper_2512_09502_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

R = 128


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_lib()


def _net():
    return wl.multi_area(seed=1234, n_areas=4, area_mean=800.0, n_ranks=R, inter_mean_indegree=150.0)


def test_128_rank_layouts_and_maps_match_oracle():
    net = _net()
    ctx = gpu_build(net)
    _, ref = oracle_layout(net)
    st = ctx.stats()
    assert st["n_synapses"] == sum(len(r["tgt"]) for r in ref["ranks"])
    assert st["n_images"] == sum(len(r["img_s"]) for r in ref["ranks"])
    for tau in range(R):
        compare_rank(ctx.get_connections(tau), ref["ranks"][tau])
    compare_maps(ctx, ref, R)
    fan_out = max(int(np.max(np.diff(ref["TP"][sig][0]), initial=0)) for sig in range(R))
    assert fan_out >= 100          # sources whose images sit on most of the other ranks
    ctx.destroy()


def _sim_net():
    """The same connectivity with power-of-two constant weights (8 pA, -64 pA) and V0
    spread over [0, 19.9) mV.  Sums of such weights are exact in fp32 whatever the order
    of the atomic additions, so both exchange schemes must give identical trajectories;
    the sources, targets and delays do not depend on the weights (separate words of the
    synapse's Philox block)."""
    net = _net()
    prm = dataclasses.replace(wl.BALANCED_PARAMS, V_init_lo=0.0, V_init_hi=19.9, v_init_seed=6)
    net.populations = [dataclasses.replace(p, params=prm) for p in net.populations]
    net.projections = [dataclasses.replace(pr, weight=wl.Dist(wl.W_CONST, 8.0 if pr.weight.mean > 0 else -64.0))
                       for pr in net.projections]
    net.drives = [wl.Drive(0, net.n_neurons, 12000.0, wl.J_E, 1234)]
    return net


def _by_step(st, gid, steps):
    out = [[] for _ in range(steps)]
    for s, g in zip(st.tolist(), gid.tolist()):
        out[s].append(g)
    return [sorted(x) for x in out]


def test_128_rank_graph_steps_route_through_the_maps():
    """1,000 graph-captured steps (checkpoints every 50) under point-to-point and
    collective exchange give bit-identical spikes and membrane potentials.  A third run
    steps one at a time beside the single-rank FP64 oracle: V within 1e-4 mV of the
    oracle's after every step until the first step whose spikes differ, and that
    difference must be a threshold decision taken in the two precisions -- each neuron
    that spiked on one side only sits within 1e-4 mV of V_th on the side where it did
    not.  The stepwise run equals the graph-captured one at every checkpoint it
    reaches."""
    net = _sim_net()
    steps, chunk = 1000, 50
    runs = {}
    for exchange in ("p2p", "collective"):
        ctx = gpu_build(net, exchange=exchange, use_graph=True, spike_log_capacity=1 << 20)
        vs = []
        for _ in range(steps // chunk):
            ctx.simulate(chunk)
            vs.append(ctx.get_state(0, net.n_neurons)[0])
        st, gid = ctx.get_spikes()
        runs[exchange] = (np.stack(vs), _by_step(st, gid, steps), ctx.stats())
        ctx.destroy()
    (va, sa, xa), (vb, sb, xb) = runs["p2p"], runs["collective"]
    assert sa == sb
    np.testing.assert_array_equal(va, vb)
    assert xa["n_spikes"] == xb["n_spikes"] > 0 and xa["n_events"] == xb["n_events"] > 0

    syn = oc.generate(net)
    rk = ol.build_all(syn, ol.round_robin(net.n_neurons, 1))["ranks"][0]
    sim = on.Simulator(net, rk["row_ptr"], rk["tgt"], rk["d"], rk["w"], on.ring_slots_for(oc.max_delay(net)),
                       stored_fp32=True)
    v_th = wl.BALANCED_PARAMS.V_th
    ctx = gpu_build(net, exchange="p2p", use_graph=False, spike_log_capacity=1 << 20)
    first_diff, n_seen = None, 0
    for n in range(steps):
        ctx.simulate(1)
        vg = ctx.get_state(0, net.n_neurons)[0]
        so = set(sim.step().tolist())
        st, gid = ctx.get_spikes()
        sg = set(gid[st == n].tolist())
        if (n + 1) % chunk == 0:
            np.testing.assert_array_equal(vg, va[n // chunk])      # the stepwise run is the graph run
        n_seen += len(so)
        if so != sg:
            first_diff = n
            flipped = so ^ sg
            assert len(flipped) <= 3, (n, sorted(flipped))
            for j in flipped:
                v_side = vg[j] if j in so else sim.V[j]            # the side without the spike
                assert abs(v_side - v_th) <= 1e-4, (n, j, float(v_side))
            same = np.array(sorted(set(range(net.n_neurons)) - flipped))
            assert np.max(np.abs(vg[same] - sim.V[same])) <= 1e-4, n
            break
        assert np.max(np.abs(vg - sim.V)) <= 1e-4, n
    ctx.destroy()
    assert n_seen > 0
    first_spike = next(n for n in range(steps) if sa[n])
    assert first_diff is None or first_diff >= first_spike + 3     # delivered input entered V first
