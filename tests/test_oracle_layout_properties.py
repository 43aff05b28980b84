"""Invariants of the oracle's per-rank layout and maps on seeded random small networks
(no GPU): every rule, uneven populations, 1 to 6 logical ranks, flagged and all-sources
images.  Each network checks
  * partition invariance: the ranks' connections are exactly the generated ones;
  * the layout order: (local-first source rank, source, delay), ties in generation order;
  * images: every used remote source, plus the forced ones of the threshold xi, and an
    image row is empty exactly when its source has no connection on that rank;
  * Eq. mapalign (S = R), Eq. sortedmaps (R ascending), L = M_tau + position;
  * T / P the inverse of the R maps, H the sorted union, I the image of H[j] or -1;
  * routing: spikes routed point-to-point (T/P -> L) and collectively (Q -> I) through the
    image rows deliver exactly what every synapse of the spiking sources delivers."""
import numpy as np
import pytest

from oracle import connect as oc
from oracle import layout as ol
from paper_2512_09502_gb300 import workloads as wl

RULES = [wl.RULE_FIXED_INDEGREE, wl.RULE_FIXED_TOTAL, wl.RULE_PAIRWISE_BERNOULLI,
         wl.RULE_PAIRWISE_BERNOULLI_GEOMETRIC, wl.RULE_ONE_TO_ONE, wl.RULE_ALL_TO_ALL]


def _random_net(rng, R):
    sizes = [int(x) for x in rng.integers(3, 40, size=int(rng.integers(2, 5)))]
    firsts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int)
    pops = [wl.Population(n) for n in sizes]
    projs = []
    for _ in range(int(rng.integers(2, 7))):
        a, b = (int(x) for x in rng.integers(0, len(sizes), size=2))
        ns, nt = sizes[a], sizes[b]
        kind = RULES[int(rng.integers(0, len(RULES)))]
        if kind == wl.RULE_ONE_TO_ONE and ns != nt:
            kind = wl.RULE_ALL_TO_ALL
        param = {wl.RULE_FIXED_INDEGREE: int(rng.integers(1, 6)),
                 wl.RULE_FIXED_TOTAL: int(rng.integers(1, ns * nt // 3 + 2)),
                 wl.RULE_PAIRWISE_BERNOULLI: float(rng.uniform(0.0, 0.4)),
                 wl.RULE_PAIRWISE_BERNOULLI_GEOMETRIC: float(rng.uniform(0.02, 0.5)),
                 wl.RULE_ONE_TO_ONE: 0, wl.RULE_ALL_TO_ALL: 0}[kind]
        sign = 1.0 if rng.random() < 0.7 else -1.0
        w = wl.Dist(wl.W_NORMAL_SIGN, sign * float(rng.uniform(10, 90)), float(rng.uniform(0, 10)))
        d = wl.DELAY_NORMAL if rng.random() < 0.6 else wl.Dist(wl.D_CONST, float(rng.uniform(0.1, 3.0)))
        projs.append(wl.Projection(int(firsts[a]), ns, int(firsts[b]), nt, wl.Rule(kind, param), w, d,
                                   int(rng.integers(1, 10_000))))
    return wl.Network("random", pops, projs, n_ranks=R)


def _check(net, xi):
    R = net.n_ranks
    syn = oc.generate(net)
    part = ol.round_robin(net.n_neurons, R)
    forced = ol.forced_images(net, part, xi)
    out = ol.build_all(syn, part, forced)
    rank_of, local_of = part["rank_of"], part["local_of"]
    M = out["M"]

    # partition invariance
    flat = ol.flatten(out["ranks"], part)
    ref = np.stack([syn["src"], syn["tgt"], syn["d"]], axis=1)
    np.testing.assert_array_equal(flat[np.lexsort(flat.T[::-1])], ref[np.lexsort(ref.T[::-1])])

    for tau, rk in enumerate(out["ranks"]):
        # layout order over the whole rank: slot, source, delay, generation index
        slot = ol.source_slot(rank_of[rk["src"]], tau)
        key = np.stack([slot, local_of[rk["src"]], rk["d"], rk["gidx"]], axis=1)
        assert all(tuple(key[i]) < tuple(key[i + 1]) for i in range(len(key) - 1))
        # rows hold their own sources: local rows first, then the images
        rp = rk["row_ptr"]
        for s in range(M[tau]):
            assert np.all(rk["src"][rp[s]:rp[s + 1]] == s * R + tau)
        used = {(int(rank_of[g]), int(local_of[g])) for g in rk["src"] if rank_of[g] != tau}
        imgs = list(zip(rk["img_sigma"].tolist(), rk["img_s"].tolist()))
        assert set(imgs) == used | set(forced[tau])
        for i, (sig, s) in enumerate(imgs):
            a, b = rp[M[tau] + i], rp[M[tau] + i + 1]
            assert (b > a) == ((sig, s) in used)
            assert np.all(rk["src"][a:b] == s * R + sig)
        # Eq. sortedmaps, Eq. mapalign, L values
        Ls = []
        for sig in range(R):
            if sig == tau:
                continue
            assert np.all(np.diff(rk["R"][sig]) > 0)
            np.testing.assert_array_equal(out["S"][sig][tau], rk["R"][sig])
            Ls.append(rk["L"][sig])
        if Ls:
            Ls = np.concatenate(Ls)
            np.testing.assert_array_equal(np.sort(Ls), M[tau] + np.arange(len(Ls)))

    for sig in range(R):
        ptr, T, P = out["TP"][sig]
        for s in range(M[sig]):
            for j in range(ptr[s], ptr[s + 1]):
                assert out["ranks"][T[j]]["R"][sig][P[j]] == s
        H = out["H"][sig]
        assert np.all(np.diff(H) > 0)
        for tau in range(R):
            I = out["I"][(sig, tau)]
            if tau == sig:
                assert np.all(I < 0)
                continue
            rk = out["ranks"][tau]
            has = np.isin(H, rk["R"][sig])
            assert np.all((I >= 0) == has)
            np.testing.assert_array_equal(I[has], rk["L"][sig][np.searchsorted(rk["R"][sig], H[has])])

    # routing: point-to-point and collective delivery equal direct delivery
    rng = np.random.default_rng(net.n_neurons * 7 + R)
    spiking = np.nonzero(rng.random(net.n_neurons) < 0.3)[0]
    D = 1 << int(max(1, oc.max_delay(net))).bit_length()
    n = 5
    direct = np.zeros((D, 2, net.n_neurons))
    for e in np.nonzero(np.isin(syn["src"], spiking))[0]:
        direct[(n + syn["d"][e]) % D, 1 if syn["w"][e] < 0 else 0, syn["tgt"][e]] += syn["w"][e]
    gid_of = {(int(rank_of[g]), int(local_of[g])): g for g in range(net.n_neurons)}
    for scheme in ("p2p", "collective"):
        got = np.zeros_like(direct)
        for tau, rk in enumerate(out["ranks"]):
            rows = [int(local_of[g]) for g in spiking if rank_of[g] == tau]        # local rows
            for sig in range(R):
                if sig == tau:
                    continue
                mine = [int(local_of[g]) for g in spiking if rank_of[g] == sig]
                if scheme == "p2p":
                    pos = ol.route_p2p(mine, out["TP"][sig]).get(tau, [])
                    rows += ol.receive_p2p(pos, rk["L"][sig])
                else:
                    pos = ol.route_collective(mine, out["GQ"][sig])
                    rows += ol.receive_collective(pos, out["I"][(sig, tau)])
            ring = ol.deliver_rows(rows, rk["row_ptr"], rk["tgt"], rk["d"], rk["w"], n, D, M[tau])
            for t in range(M[tau]):
                got[:, :, gid_of[(tau, t)]] += ring[:, :, t]
        np.testing.assert_allclose(got, direct, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("seed", range(30))
def test_random_networks(seed):
    rng = np.random.default_rng(1000 + seed)
    R = int(rng.integers(1, 7))
    xi = [0.0, 0.5, 1.0][seed % 3]
    _check(_random_net(rng, R), xi)
