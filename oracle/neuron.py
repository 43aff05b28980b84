"""iaf_psc_exp exact integration and ring-buffer spike delivery (oracle; test
infrastructure only).

The paper does not state neuron equations; its networks are current-based point
neurons (Results, "Collective communication: scalable balanced network").  The model
here is the leaky integrate-and-fire neuron with exponentially decaying synaptic
currents, integrated exactly on the time grid (Rotter & Diesmann 1999):

    P22 = exp(-h/tau_m),  P11 = exp(-h/tau_syn),
    P20 = -(tau_m / C_m) expm1(-h/tau_m),
    P21 = (1/C_m) exp(-h/tau_m) (-expm1(-h delta)) / delta,  delta = 1/tau_syn - 1/tau_m
          (h when delta = 0: the limit tau_syn -> tau_m).

Step n of each neuron (reading; the paper is silent on the update order):
  1. not refractory: V <- P22 V + P21_ex I_ex + P21_in I_in + P20 I_e;
     refractory: the counter decreases and V stays at V_reset;
  2. I_x <- P11_x I_x + ring[n mod D][x]; the slot is cleared; a Poisson drive adds
     k J with k drawn from the Poisson table: word (gid mod 4) of the POISSON-stream
     block with counter (gid div 4, n), so four consecutive neurons share one block;
  3. V >= V_th: V <- V_reset, refractory for round(t_ref / h) steps, spike (n, gid).
Spike delivery (Appendix, point-to-point example, delivery figure): a spike of step n
through a connection of delay d (>= 1 step) and weight w adds w to slot (n + d) mod D
of the target's ring for receptor ex (w >= 0) or in (w < 0).

Reading: the method computes the propagators in FP64 and stores them in FP32; the
simulator can take them that way (``stored_fp32``), which is what network-level
comparisons use -- the balanced networks are chaotic, so a 3e-8 relative change of a
constant alone moves 1-s population rates by several percent.

Pinned by tests/test_oracle_neuron.py: the closed-form PSP at grid points, the
steady state and the closed-form inter-spike interval under constant current, the
tau_syn -> tau_m limit, and the delivery slots of the worked example.
"""
from __future__ import annotations

import math

import numpy as np

from . import philox as ph
from . import sampling as sm


def propagators(p, h: float):
    """FP64 propagators of one parameter set (dict with P22, P20, P11/P21 per receptor)."""
    P22 = math.exp(-h / p.tau_m)
    P20 = -(p.tau_m / p.C_m) * math.expm1(-h / p.tau_m)
    out = dict(P22=P22, P20=P20)
    for x, ts in (("ex", p.tau_syn_ex), ("in", p.tau_syn_in)):
        out["P11_" + x] = math.exp(-h / ts)
        delta = 1.0 / ts - 1.0 / p.tau_m
        if delta == 0.0:
            frac = h
        else:
            frac = -math.expm1(-h * delta) / delta
        out["P21_" + x] = (1.0 / p.C_m) * P22 * frac
    out["ref_steps"] = int(round(p.t_ref / h))
    return out


def psp_closed_form(J: float, p, t):
    """Membrane response to one current jump J at t = 0 (tau_syn != tau_m)."""
    ts, tm = p.tau_syn_ex, p.tau_m
    return (J / p.C_m) * ts * tm / (tm - ts) * (np.exp(-t / tm) - np.exp(-t / ts))


def initial_v(net):
    """V0 per neuron: lo, or lo + (hi - lo) u01 from stream VINIT (counter gid,
    word2 = population index) when hi > lo."""
    out = []
    first = 0
    for pi, pop in enumerate(net.populations):
        prm = pop.params
        g = np.arange(first, first + pop.n, dtype=np.uint64)
        if prm.V_init_hi > prm.V_init_lo:
            b = ph.stream(g, pi, ph.PURPOSE_VINIT, prm.v_init_seed)
            out.append(prm.V_init_lo + (prm.V_init_hi - prm.V_init_lo) * sm.u01(b[0]))
        else:
            out.append(np.full(pop.n, float(prm.V_init_lo)))
        first += pop.n
    return np.concatenate(out) if out else np.zeros(0)


class Simulator:
    """Plain per-step simulation over a global source-sorted layout (rows = gids)."""

    def __init__(self, net, row_ptr, tgt, d, w, ring_slots: int, stored_fp32: bool = False):
        """``stored_fp32``: use the propagators as the method stores them -- computed
        in FP64, rounded once to FP32 (like the stored weights).  The membrane and
        current arithmetic stays FP64 either way."""
        self.net = net
        self.N = net.n_neurons
        self.h = net.dt
        self.row_ptr, self.tgt, self.d, self.w = row_ptr, tgt, d, w
        self.D = ring_slots
        fields = ["P22", "P20", "P11_ex", "P11_in", "P21_ex", "P21_in"]
        per = {f: [] for f in fields + ["I_e", "V_th", "V_reset", "ref_steps"]}
        for pop in net.populations:
            pr = propagators(pop.params, self.h)
            for f in fields:
                v = float(np.float32(pr[f])) if stored_fp32 else pr[f]
                per[f].append(np.full(pop.n, v))
            per["ref_steps"].append(np.full(pop.n, pr["ref_steps"], dtype=np.int64))
            per["I_e"].append(np.full(pop.n, pop.params.I_e))
            per["V_th"].append(np.full(pop.n, pop.params.V_th))
            per["V_reset"].append(np.full(pop.n, pop.params.V_reset))
        self.c = {k: np.concatenate(v) for k, v in per.items()}
        self.V = initial_v(net)
        self.Iex = np.zeros(self.N)
        self.Iin = np.zeros(self.N)
        self.refr = np.zeros(self.N, dtype=np.int64)
        self.ring = np.zeros((self.D, 2, self.N))
        self.step_no = 0
        self.drives = [(dr, sm.poisson_table(dr.rate_hz, self.h)) for dr in net.drives]

    def step(self):
        n, c = self.step_no, self.c
        free = self.refr == 0
        v_new = c["P22"] * self.V + c["P21_ex"] * self.Iex + c["P21_in"] * self.Iin + c["P20"] * c["I_e"]
        self.V = np.where(free, v_new, self.V)
        self.refr = np.where(free, self.refr, self.refr - 1)
        slot = n % self.D
        self.Iex = c["P11_ex"] * self.Iex + self.ring[slot, 0]
        self.Iin = c["P11_in"] * self.Iin + self.ring[slot, 1]
        self.ring[slot] = 0.0
        for di, (dr, thr) in enumerate(self.drives):
            k = poisson_counts(thr, di, dr.seed, dr.first, dr.n, n)
            if dr.weight >= 0:
                self.Iex[dr.first:dr.first + dr.n] += k * dr.weight
            else:
                self.Iin[dr.first:dr.first + dr.n] += k * dr.weight
        spk = np.nonzero(self.V >= c["V_th"])[0]
        self.V[spk] = c["V_reset"][spk]
        self.refr[spk] = c["ref_steps"][spk]
        self.deliver(n, spk)
        self.step_no += 1
        return spk

    def deliver(self, n, spikes):
        for g in spikes:
            a, b = self.row_ptr[g], self.row_ptr[g + 1]
            if a == b:
                continue
            slots = (n + self.d[a:b]) % self.D
            rec = (self.w[a:b] < 0).astype(np.int64)
            np.add.at(self.ring, (slots, rec, self.tgt[a:b]), self.w[a:b])

    def run(self, steps: int, record_v: bool = False):
        spikes, vs = [], []
        for _ in range(steps):
            n = self.step_no
            for g in self.step():
                spikes.append((n, int(g)))
            if record_v:
                vs.append(self.V.copy())
        return spikes, (np.array(vs) if record_v else None)


def poisson_counts(thr, drive_index: int, seed: int, first: int, n_neurons: int, step: int):
    """Drive counts of neurons first .. first + n_neurons - 1 at step ``step``: neuron g
    inverts word (g mod 4) of the POISSON block with counter (g div 4, step) through the
    count table ``thr``."""
    g = np.arange(first, first + n_neurons, dtype=np.uint64)
    ctr = (g >> np.uint64(2)) | (np.uint64(step) << np.uint64(32))
    words = ph.stream(ctr, drive_index, ph.PURPOSE_POISSON, seed)
    return sm.inverse_table(thr, np.choose((g & np.uint64(3)).astype(np.int64), words))


def ring_slots_for(max_delay: int) -> int:
    """Ring length: the next power of two above the largest delay."""
    D = 1
    while D < max_delay + 1:
        D *= 2
    return D
