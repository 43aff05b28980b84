"""Pins of the oracle's per-rank layout and communication maps (no GPU)."""
import json
import os

import numpy as np
import pytest

from oracle import connect as oc
from oracle import layout as ol
from paper_2512_09502_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _syn_from_pairs(pairs, d=1, w=1.0):
    pairs = np.asarray(pairs, dtype=np.int64)
    n = len(pairs)
    return dict(src=pairs[:, 0], tgt=pairs[:, 1], d=np.full(n, d, np.int64),
                w=np.full(n, w), gidx=np.arange(n, dtype=np.int64))


def test_routing_figures_example():
    g = json.load(open(os.path.join(GOLD, "routing_figures_example.json")))
    part = ol.block_partition(g["rank_sizes"])
    out = ol.build_all(_syn_from_pairs(g["connections_global"]), part)
    ptr, T, P = out["TP"][2]
    assert T[ptr[0]:ptr[1]].tolist() == g["T_2_0"]
    assert P[ptr[0]:ptr[1]].tolist() == g["P_2_0"]
    # neuron 1 of rank 0 -> image 2 of rank 1
    pk = ol.route_p2p([1], out["TP"][0])
    assert ol.receive_p2p(pk[1], out["ranks"][1]["L"][0]) == [g["image_of_rank0_neuron1_in_rank1"]]
    assert [s for s in range(3) if s != 1 and len(out["ranks"][1]["R"][s])] == g["rank1_map_sources"]
    # collective: neuron 0 of rank 2 at position 0 of H_{0,2}, received by ranks 0 and 1
    q = ol.route_collective([0], out["GQ"][2])
    assert q == [g["H_2_position_of_0"]]
    recv = [tau for tau in range(3) if ol.receive_collective(q, out["I"][(2, tau)])]
    assert recv == g["collective_receivers_of_rank2_neuron0"]
    # collective and p2p reach the same images
    for sig in range(3):
        for s in range(part["M"][sig]):
            pk = ol.route_p2p([s], out["TP"][sig])
            p2p = {(tau, l) for tau, pos in pk.items() for l in ol.receive_p2p(pos, out["ranks"][tau]["L"][sig])}
            q = ol.route_collective([s], out["GQ"][sig])
            col = {(tau, l) for tau in range(3) for l in ol.receive_collective(q, out["I"][(sig, tau)])}
            assert p2p == col


def test_p2p_appendix_example():
    g = json.load(open(os.path.join(GOLD, "p2p_appendix_example.json")))
    # source side T/P tables of rank 0 (neurons 0..799)
    M0 = 800
    lists = {int(k): v for k, v in g["tp"].items()}
    ptr = np.zeros(M0 + 1, np.int64)
    T, P = [], []
    for s in range(M0):
        for tau, pos in lists.get(s, []):
            T.append(tau)
            P.append(pos)
        ptr[s + 1] = len(T)
    pk = ol.route_p2p(g["spiking"], (ptr, np.array(T), np.array(P)))
    assert {str(k): v for k, v in pk.items()} == g["packets"]
    # target side: L map of rank 1 for source rank 0
    L = np.arange(1000) + 5000
    for pos, img in g["L_1_0"].items():
        L[int(pos)] = img
    imgs = ol.receive_p2p(pk[1], L)
    assert imgs == g["images_rank1"]
    # rank 1 connections of the images, then delivery into the ring
    n_rows = 800
    rows = {int(k): v for k, v in g["rows_rank1"].items()}
    rp = np.zeros(n_rows + 1, np.int64)
    tgt, d = [], []
    for r in range(n_rows):
        for t, dd in rows.get(r, []):
            tgt.append(t)
            d.append(dd)
        rp[r + 1] = len(tgt)
    w = np.linspace(1.0, 2.0, len(tgt))
    n, D = 1000, 8
    ring = ol.deliver_rows(imgs, rp, np.array(tgt), np.array(d), w, n, D, 400, multiplicity=[3, 2])
    hit = np.argwhere(ring != 0)
    got = sorted((int(t), int((slot - n) % D)) for slot, rec, t in hit)
    assert got == sorted(tuple(x) for x in g["slots"])
    assert ring[(n + 2) % D, 0, 126] == 3 * w[0] and ring[(n + 3) % D, 0, 243] == 2 * w[2]


def _layout(R, seed=3):
    net = wl.balanced(240, 60, 30, 8, wl.DELAY_NORMAL, seed=seed)
    syn = oc.generate(net)
    part = ol.round_robin(net.n_neurons, R)
    return net, syn, part, ol.build_all(syn, part)


def test_mapalign_sortedmaps_and_L_values():
    net, syn, part, out = _layout(7)
    R, M = 7, out["M"]
    for tau in range(R):
        rk = out["ranks"][tau]
        Ls = []
        for sig in range(R):
            if sig == tau:
                continue
            Rm, Lm = rk["R"][sig], rk["L"][sig]
            np.testing.assert_array_equal(out["S"][sig][tau], Rm)        # Eq. mapalign
            assert np.all(np.diff(Rm) > 0)                                  # Eq. sortedmaps
            Ls.append(Lm)
        Ls = np.concatenate(Ls)
        np.testing.assert_array_equal(np.sort(Ls), M[tau] + np.arange(len(Ls)))
        assert len(rk["row_ptr"]) == M[tau] + len(Ls) + 1


def test_tp_inverse_and_I_rule():
    net, syn, part, out = _layout(5)
    R, M = 5, out["M"]
    for sig in range(R):
        ptr, T, P = out["TP"][sig]
        for s in range(M[sig]):
            for j in range(ptr[s], ptr[s + 1]):
                assert out["ranks"][T[j]]["R"][sig][P[j]] == s
        H = out["H"][sig]
        assert np.all(np.diff(H) > 0)
        for tau in range(R):
            I = out["I"][(sig, tau)]
            has = np.isin(H, out["ranks"][tau]["R"][sig]) if tau != sig else np.zeros(len(H), bool)
            assert np.all((I >= 0) == has)
            if tau != sig:
                rk = out["ranks"][tau]
                pos = np.searchsorted(rk["R"][sig], H[has])
                np.testing.assert_array_equal(I[has], rk["L"][sig][pos])
        gptr, G, Q = out["GQ"][sig]
        np.testing.assert_array_equal(H[Q], np.repeat(np.arange(M[sig]), np.diff(gptr)))


def test_image_rows_hold_remote_connections():
    net, syn, part, out = _layout(3)
    for tau in range(3):
        rk = out["ranks"][tau]
        M = rk["M"]
        for i, (sig, s) in enumerate(zip(rk["img_sigma"], rk["img_s"])):
            a, b = rk["row_ptr"][M + i], rk["row_ptr"][M + i + 1]
            assert b > a
            assert np.all(rk["src"][a:b] == s * 3 + sig)
        a, b = rk["row_ptr"][0], rk["row_ptr"][M]
        assert np.all(rk["src"][a:b] % 3 == tau)


# ---- all-sources images (threshold xi, Methods "Remote connections") ----

@pytest.mark.parametrize("R", [1, 3])
def test_xi_quantity_is_the_mean_connections_per_source(R):
    """The quantity compared with xi is the expected number of connections that a
    projection creates on rank tau per source: exactly the generated count on tau / n_src
    for fixed in-degree, within 5 sigma of the mean for fixed total and pairwise
    Bernoulli (their counts on every rank sum to the total)."""
    net = wl.mixed_rules(seed=5)
    syn = oc.generate(net)
    part = ol.round_robin(net.n_neurons, R)
    for pid, pr in enumerate(net.projections):
        mine = syn["proj"] == pid
        tgts = pr.tgt_first + pr.tgt_stride * np.arange(pr.n_tgt)
        n_on = np.bincount(part["rank_of"][tgts], minlength=R)
        for tau in range(R):
            n = int(np.sum(mine & (part["rank_of"][syn["tgt"]] == tau)))
            e = ol.expected_per_source(pr, n_on[tau]) * pr.n_src
            if pr.rule.kind == wl.RULE_FIXED_INDEGREE:
                assert n == e
            else:
                assert abs(n - e) <= 5 * np.sqrt(e) + 1
    got = [ol.expected_per_source(pr) >= 1.0 for pr in net.projections]
    assert got == [True, False, True, False, True, False, True, False]


def _images(rk):
    return set(zip(rk["img_sigma"].tolist(), rk["img_s"].tolist()))


@pytest.mark.parametrize("R", [3, 8])
def test_all_sources_images_extend_the_flagged_ones(R):
    """xi = 1: the images on tau are the used sources plus every source of a projection
    reaching xi that has a target on tau (brute force over the gids); extra images have
    empty rows, the connections themselves are unchanged, S stays aligned with R."""
    net = wl.mixed_rules(n_ranks=R)
    syn = oc.generate(net)
    part = ol.round_robin(net.n_neurons, R)
    flagged = ol.build_all(syn, part)
    forced = ol.forced_images(net, part, 1.0)
    full = ol.build_all(syn, part, forced)
    for tau in range(R):
        a, b = flagged["ranks"][tau], full["ranks"][tau]
        for k in ("tgt", "d", "w", "src", "gidx"):
            np.testing.assert_array_equal(a[k], b[k])
        used = _images(a)
        want = set(used)
        for pid, pr in enumerate(net.projections):
            tg = pr.tgt_first + pr.tgt_stride * np.arange(pr.n_tgt)
            n_made = int(np.sum((syn["proj"] == pid) & (syn["tgt"] % R == tau)))
            if pr.rule.kind == wl.RULE_FIXED_INDEGREE:            # exact: K per target on tau
                assert n_made == pr.rule.param * np.sum(tg % R == tau)
            if ol.expected_per_source(pr, np.sum(tg % R == tau)) < 1.0 or not np.any(tg % R == tau):
                continue
            for g in (pr.src_first + pr.src_stride * np.arange(pr.n_src)).tolist():
                if g % R != tau:
                    want.add((g % R, g // R))
        assert _images(b) == want and len(want) > len(used)
        M = b["M"]
        for i, key in enumerate(zip(b["img_sigma"].tolist(), b["img_s"].tolist())):
            n = b["row_ptr"][M + i + 1] - b["row_ptr"][M + i]
            assert (n > 0) == (key in used)
        for sig in range(R):
            if sig != tau:
                np.testing.assert_array_equal(full["S"][sig][tau], b["R"][sig])    # Eq. mapalign
                assert np.all(np.diff(b["R"][sig]) > 0)                            # Eq. sortedmaps


def test_all_sources_images_closed_form():
    """One fixed in-degree projection S -> T with K = 8 over 1,000 + 1,000 neurons on 8
    ranks (125 targets per rank: 8 x 125 / 1000 = 1 connection per source and rank): at
    xi = 1 every rank holds an image of every source on another rank (1000 - 125
    images), at xi = 1.5 only of the sources it uses (about 1 - 1/e of them)."""
    pops = [wl.Population(1000), wl.Population(1000)]
    pr = wl.Projection(0, 1000, 1000, 1000, wl.Rule(wl.RULE_FIXED_INDEGREE, 8), wl.Dist(wl.W_CONST, 1.0),
                       wl.Dist(wl.D_CONST, 1.0), 9)
    net = wl.Network("k1", pops, [pr], n_ranks=8)
    syn = oc.generate(net)
    part = ol.round_robin(net.n_neurons, 8)
    at1 = ol.build_all(syn, part, ol.forced_images(net, part, 1.0))
    at15 = ol.build_all(syn, part, ol.forced_images(net, part, 1.5))
    for tau in range(8):
        assert len(at1["ranks"][tau]["img_s"]) == 1000 - 125
        used = np.unique(syn["src"][(syn["tgt"] % 8 == tau) & (syn["src"] % 8 != tau)])
        assert len(at15["ranks"][tau]["img_s"]) == len(used) < 1000 - 125
        assert abs(len(used) - 875 * (1 - np.exp(-1))) < 5 * np.sqrt(875 * 0.25)


def test_xi_off_is_the_flagged_layout():
    net = wl.mixed_rules(n_ranks=4)
    part = ol.round_robin(net.n_neurons, 4)
    for xi in (0.0, -1.0, 1e9):
        assert all(not v for v in ol.forced_images(net, part, xi).values())


def test_all_sources_images_only_on_ranks_with_targets():
    """Targets 1003, 1011, ... (stride 8 on 8 ranks) all live on rank 3: K = 8 over 125
    targets is 1 connection per source, so rank 3 holds 875 images and no other rank
    holds any."""
    pops = [wl.Population(1000), wl.Population(1000)]
    pr = wl.Projection(0, 1000, 1003, 125, wl.Rule(wl.RULE_FIXED_INDEGREE, 8), wl.Dist(wl.W_CONST, 1.0),
                       wl.Dist(wl.D_CONST, 1.0), 9, tgt_stride=8)
    net = wl.Network("k8_rank3", pops, [pr], n_ranks=8)
    syn = oc.generate(net)
    part = ol.round_robin(net.n_neurons, 8)
    out = ol.build_all(syn, part, ol.forced_images(net, part, 1.0))
    assert [len(r["img_s"]) for r in out["ranks"]] == [0, 0, 0, 875, 0, 0, 0, 0]
