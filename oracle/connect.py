"""Connection rules in generation order (oracle; test infrastructure only).

The paper generates connections in GPU memory from a rule dictionary and a synapse
dictionary (Methods, "Creation of the remote connection structures for point-to-point
MPI communication"; rules after Senk et al. 2022: *random, fixed in-degree* and
*random, fixed total number*, with multapses and autapses allowed as in the scalable
balanced network, Results, "Collective communication: scalable balanced network").
Pairwise Bernoulli completes the rule set.

Readings (the paper does not fix the generator):

* Every draw of projection ``p`` (0-based call order) comes from Philox-4x32-10 with
  key = the projection's seed and counter (c lo32, c hi32, p, purpose), where ``c``
  is the projection-local counter:
    - fixed in-degree K:   c = (t - t_first) * K + k, for target t, k < K;
    - fixed total N:       c = j, the draw index;
    - pairwise Bernoulli:  c = q = i_t * n_src + i_s (both variants).
  Sources and targets are the projection's i-th members src_first + i * src_stride
  and tgt_first + i * tgt_stride (stride 1 for population ranges; a rank-local range
  of a round-robin partition has stride R).
* Words of the SYNAPSE block: w0 -> source index, w1 -> delay step, (w2, w3) ->
  weight.  A fixed-total draw takes its target from w0 of the FT_TARGET block.  A
  Bernoulli pair q is kept iff word (q & 3) of the PB_TEST block at counter q >> 2 is
  below floor(p 2^32) (all pairs when p = 1).  The geometric-skipping variant draws
  the gaps between kept pairs instead (``bernoulli_geometric_pairs``).
* Generation order is (projection order, c ascending).  ``gidx`` = cbase_p + c, with
  cbase_p the summed counter-space sizes (n_tgt K, N, n_tgt n_src) of earlier
  projections; it is the tie-break of the source-sorted layout.

Keyed by global ids and projection-local counters, the synapse set does not depend on
how neurons are partitioned over ranks: this is how the source-side variant of
RemoteConnect regenerates the same sources as the target side (Methods,
"Point-to-point MPI communication").

Pinned by tests/test_oracle_connect.py: exact in-degree / totals, brute-force
enumeration of a tiny Bernoulli projection, chi-square of source, target and delay
histograms, partition invariance.
"""
from __future__ import annotations

import numpy as np

from . import philox as ph
from . import sampling as sm


def counter_space(pr) -> int:
    """Size of the projection-local counter space."""
    if pr.rule.kind == "fixed_indegree":
        return int(pr.rule.param) * pr.n_tgt
    if pr.rule.kind == "fixed_total":
        return int(pr.rule.param)
    if pr.rule.kind in ("pairwise_bernoulli", "pairwise_bernoulli_geometric", "all_to_all"):
        return pr.n_tgt * pr.n_src
    if pr.rule.kind == "one_to_one":
        return pr.n_tgt
    raise ValueError(pr.rule.kind)


def counter_bases(net):
    out, acc = [], 0
    for pr in net.projections:
        out.append(acc)
        acc += counter_space(pr)
    return out, acc


def bernoulli_threshold(p: float) -> int:
    """Keep a pair iff its word < floor(p 2^32); p = 1 keeps every pair."""
    return int(np.floor(p * 4294967296.0))


def projection_synapses(net, pid: int, counters=None):
    """All synapses of projection ``pid`` (or those with the given counters, for
    fixed in-degree / fixed total) in generation order.

    Returns dict of arrays: src, tgt (global ids), d (steps), w (fp64), c (counter)."""
    pr = net.projections[pid]
    kind = pr.rule.kind
    if kind == "fixed_indegree":
        K = int(pr.rule.param)
        c = np.arange(pr.n_tgt * K, dtype=np.uint64) if counters is None else np.asarray(counters, np.uint64)
        t_local = (c // np.uint64(K)).astype(np.int64)
        b = ph.stream(c, pid, ph.PURPOSE_SYNAPSE, pr.seed)
        src = pr.src_first + pr.src_stride * sm.uniform_index(b[0], pr.n_src).astype(np.int64)
        tgt = pr.tgt_first + pr.tgt_stride * t_local
    elif kind == "one_to_one":
        # target i connects from source i (the two sets have the same size); counter c = i
        if pr.n_src != pr.n_tgt:
            raise ValueError("one-to-one needs as many sources as targets")
        c = np.arange(pr.n_tgt, dtype=np.uint64) if counters is None else np.asarray(counters, np.uint64)
        b = ph.stream(c, pid, ph.PURPOSE_SYNAPSE, pr.seed)
        src = pr.src_first + pr.src_stride * c.astype(np.int64)
        tgt = pr.tgt_first + pr.tgt_stride * c.astype(np.int64)
    elif kind == "all_to_all":
        # every (target i_t, source i_s) pair once, counter c = i_t n_src + i_s
        c = (np.arange(pr.n_tgt * pr.n_src, dtype=np.uint64) if counters is None
             else np.asarray(counters, np.uint64))
        b = ph.stream(c, pid, ph.PURPOSE_SYNAPSE, pr.seed)
        src = pr.src_first + pr.src_stride * (c % np.uint64(pr.n_src)).astype(np.int64)
        tgt = pr.tgt_first + pr.tgt_stride * (c // np.uint64(pr.n_src)).astype(np.int64)
    elif kind == "fixed_total":
        N = int(pr.rule.param)
        c = np.arange(N, dtype=np.uint64) if counters is None else np.asarray(counters, np.uint64)
        b = ph.stream(c, pid, ph.PURPOSE_SYNAPSE, pr.seed)
        bt = ph.stream(c, pid, ph.PURPOSE_FT_TARGET, pr.seed)
        src = pr.src_first + pr.src_stride * sm.uniform_index(b[0], pr.n_src).astype(np.int64)
        tgt = pr.tgt_first + pr.tgt_stride * sm.uniform_index(bt[0], pr.n_tgt).astype(np.int64)
    elif kind == "pairwise_bernoulli_geometric":
        assert counters is None
        c = bernoulli_geometric_pairs(pr, pid)
        b = ph.stream(c, pid, ph.PURPOSE_SYNAPSE, pr.seed)
        src = pr.src_first + pr.src_stride * (c % np.uint64(pr.n_src)).astype(np.int64)
        tgt = pr.tgt_first + pr.tgt_stride * (c // np.uint64(pr.n_src)).astype(np.int64)
    elif kind == "pairwise_bernoulli":
        assert counters is None
        q = np.arange(pr.n_tgt * pr.n_src, dtype=np.uint64)
        tb = ph.stream(q >> np.uint64(2), pid, ph.PURPOSE_PB_TEST, pr.seed)
        lane = (q & np.uint64(3)).astype(np.int64)
        word = np.choose(lane, tb)
        keep = word < np.uint64(bernoulli_threshold(pr.rule.param))
        c = q[keep]
        b = ph.stream(c, pid, ph.PURPOSE_SYNAPSE, pr.seed)
        src = pr.src_first + pr.src_stride * (c % np.uint64(pr.n_src)).astype(np.int64)
        tgt = pr.tgt_first + pr.tgt_stride * (c // np.uint64(pr.n_src)).astype(np.int64)
    else:
        raise ValueError(kind)
    d = sm.delay_steps(pr.delay, net.dt, b[1], len(c))
    w = sm.weight_values(pr.weight, b[2], b[3], len(c))
    return dict(src=src, tgt=tgt, d=d, w=w, c=c.astype(np.int64))


def bernoulli_geometric_pairs(pr, pid: int):
    """Kept pairs q = i_t * n_src + i_s of pairwise Bernoulli by geometric skipping, in
    (target, source) order.  For target i_t the j-th gap G_j inverts word w0 of the
    PB_GAP block at counter i_t * n_src + j through the gap table; the kept sources are
    s_j = sum_{i <= j} (G_i + 1) - 1 while below n_src.  Each pair is kept with
    probability p, independently, as in the pair-by-pair rule, at a cost of one draw
    per kept pair (plus one) instead of one per pair."""
    p = float(pr.rule.param)
    if p == 0.0:
        return np.zeros(0, dtype=np.uint64)
    thr = sm.geometric_gap_table(p)
    out = []
    n = pr.n_src
    for ti in range(pr.n_tgt):
        ctr = np.uint64(ti * n) + np.arange(n, dtype=np.uint64)
        g = sm.inverse_table(thr, ph.stream(ctr, pid, ph.PURPOSE_PB_GAP, pr.seed)[0])
        s = np.cumsum(g + 1) - 1
        s = s[s < n]
        out.append(np.uint64(ti * n) + s.astype(np.uint64))
    return np.concatenate(out) if out else np.zeros(0, dtype=np.uint64)


def generate(net):
    """Every synapse of the network in generation order, with its ``gidx``."""
    bases, _ = counter_bases(net)
    parts = []
    for pid in range(len(net.projections)):
        s = projection_synapses(net, pid)
        s["gidx"] = bases[pid] + s["c"]
        s["proj"] = np.full(len(s["c"]), pid, dtype=np.int64)
        parts.append(s)
    keys = ["src", "tgt", "d", "w", "c", "gidx", "proj"]
    if not parts:
        return {k: np.zeros(0, np.float64 if k == "w" else np.int64) for k in keys}
    return {k: np.concatenate([p[k] for p in parts]) for k in keys}


def fixed_indegree_target(net, pid: int, t: int):
    """The K synapses of one target t of a fixed in-degree projection (sampled
    parity at sizes the full oracle cannot build)."""
    pr = net.projections[pid]
    K = int(pr.rule.param)
    i = (t - pr.tgt_first) // pr.tgt_stride
    c = np.arange(i * K, (i + 1) * K, dtype=np.uint64)
    return projection_synapses(net, pid, counters=c)


def max_delay(net) -> int:
    return max((sm.max_delay_steps(pr.delay, net.dt) for pr in net.projections), default=1)
