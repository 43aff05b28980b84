"""Seeded synthetic network descriptions shared by the tests, ``bench.py`` and the oracle.

This module only *describes* networks (population sizes, connection rules, parameter
distributions, seeds).  It holds none of the method's arithmetic: no random number is
drawn here that the construction method itself draws (sources, delays, weights and
Poisson counts all come from the counter-based generator on each side).  The only
random numbers drawn here are the workload's own meta-parameters (area sizes,
connection probabilities, inter-area distances of the multi-area stand-in), which are
inputs to both the GPU path and the oracle.

The balanced networks follow the two-population E/I model of the paper's
"Scalable balanced network" section (fixed in-degree, multapses and autapses allowed,
K_E : K_I = 4 : 1).  The multi-area network is a synthetic stand-in for the
multi-area model of the "Multi-Area Model" section (32 areas, 4 layers with an E and
an I population each, point-to-point heavy structure); the real model's data files
are not available, so sizes and connection probabilities are drawn from stated
distributions with a fixed seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

RULE_FIXED_INDEGREE = "fixed_indegree"
RULE_FIXED_TOTAL = "fixed_total"
RULE_PAIRWISE_BERNOULLI = "pairwise_bernoulli"
RULE_PAIRWISE_BERNOULLI_GEOMETRIC = "pairwise_bernoulli_geometric"
RULE_ONE_TO_ONE = "one_to_one"                 # target i <- source i (n_src == n_tgt); param unused
RULE_ALL_TO_ALL = "all_to_all"                 # every source onto every target; param unused

# weight distributions
W_CONST = "const"
W_NORMAL_SIGN = "normal_sign"      # normal(mean, sd), clamped to keep the sign of mean
# delay distributions (milliseconds)
D_CONST = "const"
D_NORMAL_MIN = "normal_min"        # normal(mean, sd), clipped below at lo, quantised to dt


@dataclass(frozen=True)
class NeuronParams:
    """iaf_psc_exp parameters: mV relative to E_L = 0, pF, ms, pA."""
    tau_m: float = 10.0
    C_m: float = 250.0
    tau_syn_ex: float = 0.5
    tau_syn_in: float = 0.5
    V_th: float = 20.0
    V_reset: float = 10.0
    t_ref: float = 2.0
    I_e: float = 0.0
    V_init_lo: float = 0.0      # V0 = lo + (hi - lo) * u01 when hi > lo, else lo
    V_init_hi: float = 0.0
    v_init_seed: int = 0


@dataclass(frozen=True)
class Population:
    n: int
    params: NeuronParams = NeuronParams()
    name: str = ""


@dataclass(frozen=True)
class Rule:
    kind: str
    param: float     # K (fixed in-degree), N (fixed total), p (pairwise Bernoulli)


@dataclass(frozen=True)
class Dist:
    kind: str
    mean: float
    sd: float = 0.0
    lo: float = 0.0


@dataclass(frozen=True)
class Projection:
    src_first: int
    n_src: int
    tgt_first: int
    n_tgt: int
    rule: Rule
    weight: Dist
    delay: Dist
    seed: int
    src_stride: int = 1     # source gids src_first + i * src_stride, i < n_src
    tgt_stride: int = 1     # target gids tgt_first + i * tgt_stride, i < n_tgt


@dataclass(frozen=True)
class Drive:
    """Independent Poisson spike trains of rate_hz, each spike adding ``weight`` pA."""
    first: int
    n: int
    rate_hz: float
    weight: float
    seed: int


@dataclass
class Network:
    name: str
    populations: List[Population]
    projections: List[Projection]
    drives: List[Drive] = field(default_factory=list)
    n_ranks: int = 1
    dt: float = 0.1

    @property
    def n_neurons(self) -> int:
        return int(sum(p.n for p in self.populations))

    def pop_ranges(self) -> List[Tuple[int, int]]:
        out, first = [], 0
        for p in self.populations:
            out.append((first, p.n))
            first += p.n
        return out

    def n_synapses_fixed(self) -> Optional[int]:
        """Exact synapse count when every rule fixes it (fixed in-degree / total)."""
        tot = 0
        for pr in self.projections:
            if pr.rule.kind == RULE_FIXED_INDEGREE:
                tot += int(pr.rule.param) * pr.n_tgt
            elif pr.rule.kind == RULE_FIXED_TOTAL:
                tot += int(pr.rule.param)
            elif pr.rule.kind == RULE_ONE_TO_ONE:
                tot += pr.n_tgt
            elif pr.rule.kind == RULE_ALL_TO_ALL:
                tot += pr.n_src * pr.n_tgt
            else:
                return None
        return tot


J_E = 87.8                     # pA
G_INH = 5.0                    # J_I = -G * J_E
BALANCED_PARAMS = NeuronParams(tau_m=10.0, C_m=250.0, tau_syn_ex=0.5, tau_syn_in=0.5,
                               V_th=20.0, V_reset=10.0, t_ref=2.0, I_e=0.0)


def balanced(n_e: int, n_i: int, k_e: int, k_i: int, delay: Dist, *, seed: int = 1234,
             name: str = "balanced", params: NeuronParams = BALANCED_PARAMS,
             drive_rate_hz: float = 8000.0, n_ranks: int = 1, j_scale: float = 1.0) -> Network:
    """Two-population balanced random network with fixed in-degree (K_E from the E
    population, K_I from the I population onto every neuron); ``j_scale`` scales the
    recurrent weights (not the drive)."""
    n = n_e + n_i
    je = J_E * j_scale
    w_e = Dist(W_NORMAL_SIGN, je, 0.1 * je)
    w_i = Dist(W_NORMAL_SIGN, -G_INH * je, 0.1 * G_INH * je)
    projs = [
        Projection(0, n_e, 0, n, Rule(RULE_FIXED_INDEGREE, k_e), w_e, delay, seed),
        Projection(n_e, n_i, 0, n, Rule(RULE_FIXED_INDEGREE, k_i), w_i, delay, seed),
    ]
    drives = [Drive(0, n, drive_rate_hz, J_E, seed)] if drive_rate_hz > 0 else []
    return Network(name, [Population(n_e, params, "E"), Population(n_i, params, "I")],
                   projs, drives, n_ranks=n_ranks)


# Poisson drive rates that put each balanced network near the paper's ~8 Hz state
# (Results, "Collective communication: scalable balanced network").  With the stated
# neuron parameters an 8 kHz x J_E drive gives V_inf = 14 mV < V_th = 20 mV and a
# silent network, so the drive is the one free parameter set to reach ~8 Hz.
DRIVE_SMALL_HZ = 10200.0
DRIVE_SCALED_HZ = 20000.0


def indegree_scaling(factor: int, neurons_at_1: int = 500_000, **kw) -> Network:
    """The balanced network with in-degree scaled up by ``factor`` and the neuron count
    and recurrent weights scaled down by it, so that synapses and the input per neuron
    (K x J) stay fixed (paper, Appendix "Scalable balanced network with different
    in-degree scale parameter"): K = (9,000 + 2,250) x factor; at factor 1 it is the
    500k-neuron workload."""
    kw.setdefault("drive_rate_hz", DRIVE_SCALED_HZ)
    n = neurons_at_1 // factor
    return balanced(n * 4 // 5, n - n * 4 // 5, 9000 * factor, 2250 * factor, DELAY_NORMAL,
                    name=f"indegree_x{factor}", j_scale=1.0 / factor, **kw)


def balanced_small(**kw) -> Network:
    """5,000 neurons, K = 400 E + 100 I, constant 1.5 ms delay, 2.5M synapses."""
    kw.setdefault("drive_rate_hz", DRIVE_SMALL_HZ)
    return balanced(4000, 1000, 400, 100, Dist(D_CONST, 1.5), name="balanced_5k", **kw)


DELAY_NORMAL = Dist(D_NORMAL_MIN, 1.5, 0.75, 0.1)


def balanced_scaled(scale: float = 1.0, **kw) -> Network:
    """400k E + 100k I neurons at scale 1, K = 9,000 E + 2,250 I (5.625G synapses),
    delays normal(1.5, 0.75) ms clipped at 0.1 ms, quantised to dt."""
    n_e, n_i = int(round(400_000 * scale)), int(round(100_000 * scale))
    kw.setdefault("drive_rate_hz", DRIVE_SCALED_HZ)
    return balanced(n_e, n_i, 9000, 2250, DELAY_NORMAL,
                    name=f"balanced_{n_e + n_i}", **kw)


MULTI_AREA_G = 10.0            # J_I = -10 J_E: E in-degree ~3,500 vs I ~500 per target
MULTI_AREA_DRIVE_HZ = 23000.0


def multi_area(seed: int = 1234, n_areas: int = 32, area_mean: float = 31250.0,
               n_ranks: int = 1, scale: float = 1.0, per_pair_indegree: bool = False,
               inter_mean_indegree: float = 1500.0, g: float = MULTI_AREA_G,
               drive_rate_hz: float = MULTI_AREA_DRIVE_HZ) -> Network:
    """Synthetic multi-area network: ``n_areas`` areas x 8 populations (E then I, 4
    layers each), area sizes lognormal (sigma 0.3, mean preserved), intra-area 8x8
    fixed-total projections with p ~ U(0.01, 0.15), 30% of ordered area pairs
    connected from the 4 E populations of the source area onto the whole target area
    with a fixed in-degree.  By default ``inter_mean_indegree`` is each neuron's total
    inter-area in-degree, split over its connected source areas; with
    ``per_pair_indegree`` it is the mean per connected pair.  Inter-area delays are
    distance / 3.5 m/s with distance ~ U(5, 50) mm and a 10% sd.  With the balanced
    network's g = 5 the E in-degree (~3,500 per target) exceeds g times the I in-degree
    (~500), so the network is either silent or saturated; g = 10 gives it an
    inhibition-dominated (balanced) regime like the paper's models."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(n_areas)
    sizes = np.rint(area_mean * scale * np.exp(0.3 * z - 0.045)).astype(np.int64)
    pops: List[Population] = []
    area_first, pop_first = [], []          # per area: first gid; per area: 8 pop firsts
    first = 0
    for a in range(n_areas):
        area_first.append(first)
        ne = int(round(0.8 * sizes[a] / 4))
        ni = int(round(0.2 * sizes[a] / 4))
        firsts = []
        for n in [ne] * 4 + [ni] * 4:
            firsts.append(first)
            pops.append(Population(n, BALANCED_PARAMS, f"A{a}"))
            first += n
        pop_first.append(firsts)
    total = first
    area_n = [sum(p.n for p in pops[8 * a:8 * a + 8]) for a in range(n_areas)]
    pop_n = [[pops[8 * a + k].n for k in range(8)] for a in range(n_areas)]

    w_e = Dist(W_NORMAL_SIGN, J_E, 0.1 * J_E)
    w_i = Dist(W_NORMAL_SIGN, -g * J_E, 0.1 * g * J_E)
    projs: List[Projection] = []
    for a in range(n_areas):
        prob = rng.uniform(0.01, 0.15, size=(8, 8))     # [target pop, source pop]
        for q in range(8):
            for p in range(8):
                k = int(round(prob[q, p] * pop_n[a][p] * pop_n[a][q]))
                projs.append(Projection(pop_first[a][p], pop_n[a][p], pop_first[a][q],
                                        pop_n[a][q], Rule(RULE_FIXED_TOTAL, k),
                                        w_e if p < 4 else w_i, DELAY_NORMAL, seed))
    conn = rng.random((n_areas, n_areas)) < 0.3          # [source area, target area]
    np.fill_diagonal(conn, False)
    dist = rng.uniform(5.0, 50.0, size=(n_areas, n_areas))
    n_in = conn.sum(axis=0)
    for b in range(n_areas):
        for a in range(n_areas):
            if not conn[a, b]:
                continue
            mean_k = inter_mean_indegree if per_pair_indegree else inter_mean_indegree / n_in[b]
            k = max(1, int(round(mean_k * np.exp(0.3 * rng.standard_normal() - 0.045))))
            d_ms = dist[a, b] / 3.5
            e_n = sum(pop_n[a][:4])
            projs.append(Projection(area_first[a], e_n, area_first[b], area_n[b],
                                    Rule(RULE_FIXED_INDEGREE, k), w_e,
                                    Dist(D_NORMAL_MIN, d_ms, 0.1 * d_ms, 0.1), seed))
    drives = [Drive(0, total, drive_rate_hz, J_E, seed)]
    return Network(f"multi_area_{total}", pops, projs, drives, n_ranks=n_ranks)


def mixed_rules(n_ranks: int = 1, seed: int = 5, drive_rate_hz: float = 16000.0) -> Network:
    """Four populations (A, B, D excitatory; C inhibitory) joined by projections of every
    rule, with expected connections per source on both sides of 1: A->B fixed in-degree
    K = 4 (3.0 per source), B->C K = 1 (0.4), C->A fixed total 200 (1.67), D->A 30
    (0.33), A->C pairwise Bernoulli p = 0.02 (2.4), B->D by geometric gaps p = 0.005
    (0.45), C->B by geometric gaps p = 0.05 (15), and A's first half -> D with
    K = 2 (0.9); figures per source over all targets, on R ranks about
    1/R of them per rank.  The workload of the all-sources image threshold xi."""
    pops = [Population(400, BALANCED_PARAMS, "A"), Population(300, BALANCED_PARAMS, "B"),
            Population(120, BALANCED_PARAMS, "C"), Population(90, BALANCED_PARAMS, "D")]
    a, b, c, d = 0, 400, 700, 820
    w_e = Dist(W_NORMAL_SIGN, J_E, 0.1 * J_E)
    w_i = Dist(W_NORMAL_SIGN, -G_INH * J_E, 0.1 * G_INH * J_E)
    projs = [
        Projection(a, 400, b, 300, Rule(RULE_FIXED_INDEGREE, 4), w_e, DELAY_NORMAL, seed),
        Projection(b, 300, c, 120, Rule(RULE_FIXED_INDEGREE, 1), w_e, DELAY_NORMAL, seed),
        Projection(c, 120, a, 400, Rule(RULE_FIXED_TOTAL, 200), w_i, DELAY_NORMAL, seed),
        Projection(d, 90, a, 400, Rule(RULE_FIXED_TOTAL, 30), w_e, DELAY_NORMAL, seed),
        Projection(a, 400, c, 120, Rule(RULE_PAIRWISE_BERNOULLI, 0.02), w_e, DELAY_NORMAL, seed),
        Projection(b, 300, d, 90, Rule(RULE_PAIRWISE_BERNOULLI_GEOMETRIC, 0.005), w_e, DELAY_NORMAL, seed),
        Projection(c, 120, b, 300, Rule(RULE_PAIRWISE_BERNOULLI_GEOMETRIC, 0.05), w_i, DELAY_NORMAL, seed),
        Projection(a, 200, d, 90, Rule(RULE_FIXED_INDEGREE, 2), w_e, DELAY_NORMAL, seed),
    ]
    drives = [Drive(0, 910, drive_rate_hz, J_E, seed)]
    return Network("mixed_rules", pops, projs, drives, n_ranks=n_ranks)


def tiny(rule: str, param: float, n_src: int = 20, n_tgt: int = 20, *, seed: int = 7,
         delay: Dist = Dist(D_NORMAL_MIN, 0.5, 0.3, 0.1), n_ranks: int = 1,
         weight: Dist = Dist(W_NORMAL_SIGN, 50.0, 10.0)) -> Network:
    """A single projection between two small populations (used for brute force)."""
    pops = [Population(n_src, BALANCED_PARAMS, "S"), Population(n_tgt, BALANCED_PARAMS, "T")]
    pr = Projection(0, n_src, n_src, n_tgt, Rule(rule, param), weight, delay, seed)
    return Network(f"tiny_{rule}", pops, [pr], [], n_ranks=n_ranks)
