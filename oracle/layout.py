"""Per-rank connection layout, image neurons and communication maps (oracle; test
infrastructure only).

Definitions followed (paper, Methods, "Remote connections"):

* Neurons are distributed over R ranks; the build uses NEST's round-robin scheme
  (Introduction): rank(g) = g mod R, local index s = g div R.  Worked examples use a
  contiguous partition with given rank sizes.
* A connection is stored on the rank of its target.  A remote source sigma != tau is
  represented on tau by an image neuron with local index >= M_tau ("image neuron",
  "Point-to-point MPI communication").  Only sources with at least one connection into
  tau get an image (the flagged variant of RemoteConnect, used for randomly drawn
  sources).
* With the paper's threshold xi (Methods, "Remote connections"), where a projection's
  expected connections per source on rank tau reach xi, the flagging is skipped there:
  all its sources get an image on tau (``forced_images``); xi <= 0 keeps flagging.
* Connections are sorted by source as the first key so that one source's outgoing
  connections are (first index, count) ("GPU memory levels"); the second key is the
  delay, and ties keep generation order (reading: stable sort, tie-break gidx).
* Image order (reading): images of tau are ordered by (sigma, s) with sigma ascending,
  L = M_tau + position in that order -- the result RemoteConnect gives when called
  once per source rank in ascending sigma.  The rows of tau are the M_tau local
  neurons, then the images.
* R_{tau,sigma} ascending, L_{tau,sigma} aligned (Eq. sortedmaps); S_{tau,sigma} is
  built on the source side from the connections' sources and equals R (Eq. mapalign).
* T_{sigma,s} / P_{sigma,s}: for each source, the target ranks holding an image
  (ascending) and the positions in the (R, L) maps ("Creation of the remote
  connection structures for point-to-point MPI communication", simulation
  preparation).
* H_{0,sigma}: sorted union of sigma's sources with connections into other ranks of
  group 0 (all ranks); I_{0,sigma,tau}[j] = L_{tau,sigma}[i] where
  R_{tau,sigma}[i] = H_{0,sigma}[j], else -1; G_{sigma,s} / Q_{sigma,s}: the groups of
  s and its position in H ("Creation of the remote connection structures for
  collective MPI communication").

Pinned by tests/test_oracle_layout.py: the worked examples of Fig. 1, Fig. 2 and the
point-to-point appendix, Eq. mapalign / Eq. sortedmaps, the I = -1 rule, T/P
inverse consistency, exact partition invariance of the flattened synapse multiset.
"""
from __future__ import annotations

import numpy as np


def round_robin(n_neurons: int, R: int):
    """Round-robin partition: rank(g) = g mod R, local index g div R."""
    g = np.arange(n_neurons, dtype=np.int64)
    return dict(rank_of=g % R, local_of=g // R, M=[(n_neurons - t + R - 1) // R for t in range(R)], R=R)


def block_partition(sizes):
    """Contiguous partition with the given rank sizes (worked examples)."""
    sizes = list(sizes)
    rank_of = np.repeat(np.arange(len(sizes)), sizes).astype(np.int64)
    local_of = np.concatenate([np.arange(m) for m in sizes]).astype(np.int64) if sizes else np.zeros(0, np.int64)
    return dict(rank_of=rank_of, local_of=local_of, M=sizes, R=len(sizes))


def source_slot(sigma, tau):
    """Order of source ranks seen from tau: local first (0), then sigma ascending."""
    sigma = np.asarray(sigma)
    return np.where(sigma == tau, 0, np.where(sigma < tau, sigma + 1, sigma))


def expected_per_source(pr, n_tgt_on=None) -> float:
    """Expected connections per source that a projection creates on one rank holding
    ``n_tgt_on`` of its targets (default: all of them), the ratio the paper's xi
    heuristic compares (Methods, "Remote connections": K_in N_target / N_source for the
    fixed in-degree rule, N_target the targets on the target process): K n_on / n_src
    (fixed in-degree), N n_on / (n_tgt n_src) (fixed total, N spread uniformly over
    the targets), p n_on (pairwise Bernoulli)."""
    n_on = pr.n_tgt if n_tgt_on is None else int(n_tgt_on)
    if pr.rule.kind in ("one_to_one", "all_to_all"):
        # rules that use every source of the call need no flagging decision: the
        # flagged images are the used ones (Methods, "Remote connections")
        return 0.0
    if pr.rule.kind == "fixed_indegree":
        return pr.rule.param * n_on / pr.n_src
    if pr.rule.kind == "fixed_total":
        return pr.rule.param * n_on / (pr.n_tgt * pr.n_src)
    return pr.rule.param * n_on                        # pairwise Bernoulli (both variants)


def forced_images(net, part, xi: float):
    """All-sources variant (xi > 0): where a projection's expected connections per source
    on rank tau reach xi, every one of its sources on another rank gets an image on tau,
    whether or not it is used there.  Returns {tau: set of (sigma, s)}; empty sets for
    xi <= 0 (flagged images only)."""
    R = part["R"]
    out = {t: set() for t in range(R)}
    if xi <= 0:
        return out
    rank_of, local_of = part["rank_of"], part["local_of"]
    for pr in net.projections:
        srcs = pr.src_first + pr.src_stride * np.arange(pr.n_src)
        tgts = pr.tgt_first + pr.tgt_stride * np.arange(pr.n_tgt)
        n_on = np.bincount(rank_of[tgts], minlength=R)
        for tau in range(R):
            if n_on[tau] == 0 or expected_per_source(pr, n_on[tau]) < xi:
                continue
            for g in srcs:
                if rank_of[g] != tau:
                    out[tau].add((int(rank_of[g]), int(local_of[g])))
    return out


def build_rank(syn, part, tau: int, forced=()):
    """Connections of rank tau, sorted by (local-first source rank, source, delay),
    ties in generation order.  Returns dict with row_ptr (M_tau + n_img + 1), tgt
    (local target index), d, w, src (global), gidx, img_sigma / img_s per image row
    and the R / L maps per source rank.  ``forced`` adds images (sigma, s) without
    connections (the all-sources variant); their rows are empty."""
    R, M = part["R"], part["M"]
    rank_of, local_of = part["rank_of"], part["local_of"]
    sel = np.nonzero(rank_of[syn["tgt"]] == tau)[0]
    src = syn["src"][sel]
    sigma = rank_of[src]
    s = local_of[src]
    sp = source_slot(sigma, tau)
    order = np.lexsort((syn["gidx"][sel], syn["d"][sel], s, sp))
    sel, src, sigma, s, sp = sel[order], src[order], sigma[order], s[order], sp[order]
    local = sp == 0
    local_counts = np.bincount(s[local], minlength=M[tau]).astype(np.int64)
    rs, rsig = s[~local], sigma[~local]
    if len(rs):
        new_run = np.ones(len(rs), dtype=bool)
        new_run[1:] = (rs[1:] != rs[:-1]) | (rsig[1:] != rsig[:-1])
        starts = np.nonzero(new_run)[0]
        img_counts = np.diff(np.append(starts, len(rs)))
        img_sigma, img_s = rsig[starts], rs[starts]
    else:
        img_counts = np.zeros(0, np.int64)
        img_sigma = img_s = np.zeros(0, np.int64)
    if forced:
        # union with the forced images, in (sigma, s) order; forced-only rows are empty
        have = dict(zip(zip(img_sigma.tolist(), img_s.tolist()), img_counts.tolist()))
        keys = sorted(set(have) | set(forced))
        img_sigma = np.array([k[0] for k in keys], dtype=np.int64)
        img_s = np.array([k[1] for k in keys], dtype=np.int64)
        img_counts = np.array([have.get(k, 0) for k in keys], dtype=np.int64)
    row_ptr = np.concatenate([[0], np.cumsum(np.concatenate([local_counts, img_counts]))]).astype(np.int64)
    maps_R, maps_L = {}, {}
    for sig in range(R):
        if sig == tau:
            continue
        m = img_sigma == sig
        maps_R[sig] = img_s[m].astype(np.int64)
        maps_L[sig] = (M[tau] + np.nonzero(m)[0]).astype(np.int64)
    return dict(row_ptr=row_ptr, tgt=local_of[syn["tgt"][sel]].astype(np.int64),
                d=syn["d"][sel].astype(np.int64), w=syn["w"][sel], src=src,
                gidx=syn["gidx"][sel], img_sigma=img_sigma.astype(np.int64),
                img_s=img_s.astype(np.int64), R=maps_R, L=maps_L, M=M[tau])


def source_sequences(syn, part, sigma: int, forced=None):
    """Source side: S_{tau,sigma} for every tau != sigma, from the sources of the
    connections whose source lives on sigma (no access to tau's maps), plus the forced
    images of the all-sources variant (known on sigma from the projection alone)."""
    rank_of, local_of = part["rank_of"], part["local_of"]
    src, tgt = syn["src"], syn["tgt"]
    mine = rank_of[src] == sigma
    out = {}
    for tau in range(part["R"]):
        if tau == sigma:
            continue
        m = mine & (rank_of[tgt] == tau)
        used = local_of[src[m]]
        extra = [s for (sg, s) in (forced or {}).get(tau, ()) if sg == sigma]
        out[tau] = np.unique(np.concatenate([used, np.array(extra, dtype=np.int64)])).astype(np.int64)
    return out


def tp_tables(S_of_sigma, M_sigma: int, R: int, sigma: int):
    """T_{sigma,s}, P_{sigma,s} for s < M_sigma as CSR (ptr, T, P), built by walking
    every S_{tau,sigma} in ascending tau and appending (tau, i) to s's lists."""
    lists = [[] for _ in range(M_sigma)]
    for tau in range(R):
        if tau == sigma:
            continue
        for i, s in enumerate(S_of_sigma[tau]):
            lists[int(s)].append((tau, i))
    ptr = np.zeros(M_sigma + 1, dtype=np.int64)
    T, P = [], []
    for s in range(M_sigma):
        for tau, i in lists[s]:
            T.append(tau)
            P.append(i)
        ptr[s + 1] = len(T)
    return ptr, np.array(T, dtype=np.int64), np.array(P, dtype=np.int64)


def host_array(S_of_sigma, R: int, sigma: int):
    """H_{0,sigma}: sorted union of sigma's sources with an image in another rank."""
    parts = [S_of_sigma[t] for t in range(R) if t != sigma]
    if not parts:
        return np.zeros(0, np.int64)
    return np.unique(np.concatenate(parts)).astype(np.int64)


def image_array(H, R_map, L_map):
    """I_{0,sigma,tau}: L of H[j] in tau's map when R contains it, else -1."""
    out = np.full(len(H), -1, dtype=np.int64)
    for j, h in enumerate(H):
        i = np.searchsorted(R_map, h)
        if i < len(R_map) and R_map[i] == h:
            out[j] = L_map[i]
    return out


def gq_tables(H, M_sigma: int):
    """G_{sigma,s}, Q_{sigma,s} for the single group 0 as CSR (ptr, G, Q)."""
    cnt = np.zeros(M_sigma, dtype=np.int64)
    cnt[H] = 1
    ptr = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    return ptr, np.zeros(len(H), np.int64), np.arange(len(H), dtype=np.int64)


def build_all(syn, part, forced=None):
    """Every rank's layout and every map (``forced``: the all-sources images per rank,
    see forced_images)."""
    R, M = part["R"], part["M"]
    forced = forced or {t: set() for t in range(R)}
    ranks = [build_rank(syn, part, tau, forced.get(tau, ())) for tau in range(R)]
    S = [source_sequences(syn, part, sig, forced) for sig in range(R)]
    TP = [tp_tables(S[sig], M[sig], R, sig) for sig in range(R)]
    H = [host_array(S[sig], R, sig) for sig in range(R)]
    I = {}
    for sig in range(R):
        for tau in range(R):
            if tau != sig:
                I[(sig, tau)] = image_array(H[sig], ranks[tau]["R"][sig], ranks[tau]["L"][sig])
            else:
                I[(sig, tau)] = np.full(len(H[sig]), -1, dtype=np.int64)
    GQ = [gq_tables(H[sig], M[sig]) for sig in range(R)]
    return dict(M=M, ranks=ranks, S=S, TP=TP, H=H, I=I, GQ=GQ, part=part)


def flatten(ranks, part):
    """Global (src, tgt, d) triples of every rank (targets back to global ids)."""
    R = part["R"]
    gid_of = np.zeros((R, max(part["M"]) if part["M"] else 0), dtype=np.int64)
    gid_of[part["rank_of"], part["local_of"]] = np.arange(len(part["rank_of"]))
    out = []
    for tau, rk in enumerate(ranks):
        out.append(np.stack([rk["src"], gid_of[tau][rk["tgt"]], rk["d"]], axis=1))
    return np.concatenate(out) if out else np.zeros((0, 3), np.int64)


def route_p2p(spiking_local, TP_sigma):
    """Point-to-point routing on the source side (Appendix, point-to-point example):
    for each spiking local source s of sigma, one (tau, position) packet entry per
    element of T_{sigma,s} / P_{sigma,s}.  Returns {tau: [positions]} in spike order."""
    ptr, T, P = TP_sigma
    packets = {}
    for s in spiking_local:
        for j in range(ptr[s], ptr[s + 1]):
            packets.setdefault(int(T[j]), []).append(int(P[j]))
    return packets


def receive_p2p(positions, L_map):
    """Target side: map received positions to local image indices via L_{tau,sigma}."""
    return [int(L_map[i]) for i in positions]


def route_collective(spiking_local, GQ_sigma):
    """Collective routing: positions Q_{sigma,s} in H_{0,sigma} of the spiking sources
    that belong to group 0 (the payload every rank of the group receives)."""
    ptr, G, Q = GQ_sigma
    out = []
    for s in spiking_local:
        for j in range(ptr[s], ptr[s + 1]):
            out.append(int(Q[j]))
    return out


def receive_collective(positions, I_sigma_tau):
    """Rank tau keeps the positions whose I_{0,sigma,tau} entry is not -1."""
    return [int(I_sigma_tau[q]) for q in positions if I_sigma_tau[q] >= 0]


def deliver_rows(rows, row_ptr, tgt, d, w, n: int, D: int, n_local: int, multiplicity=None):
    """Ring-buffer contributions of spikes through whole rows (Appendix, delivery
    figure): slot (n + d) mod D of each target receives multiplicity * w.
    Returns a dense (D, 2, n_local) array of contributions."""
    ring = np.zeros((D, 2, n_local))
    for k, r in enumerate(rows):
        m = 1 if multiplicity is None else multiplicity[k]
        for e in range(row_ptr[r], row_ptr[r + 1]):
            ring[(n + d[e]) % D, 1 if w[e] < 0 else 0, tgt[e]] += m * w[e]
    return ring
