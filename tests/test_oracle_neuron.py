"""Pins of the oracle's iaf_psc_exp integration and ring-buffer delivery (no GPU)."""
import math

import numpy as np

from oracle import neuron as on
from paper_2512_09502_gb300 import workloads as wl


def _one_neuron_net(params, drives=()):
    return wl.Network("one", [wl.Population(1, params)], [], list(drives))


def test_psp_closed_form_on_grid():
    """A current jump J at step 0 gives V(k h) equal to the closed-form PSP."""
    p = wl.BALANCED_PARAMS
    net = _one_neuron_net(p)
    sim = on.Simulator(net, np.array([0, 0]), np.zeros(0, np.int64), np.zeros(0, np.int64),
                       np.zeros(0), 8)
    J = 87.8
    sim.ring[0, 0, 0] = J         # arrives in step 0
    _, vs = sim.run(60, record_v=True)
    t = np.arange(60) * net.dt    # after step k the neuron has integrated k steps
    ref = on.psp_closed_form(J, p, t)
    np.testing.assert_allclose(vs[:, 0], ref, rtol=0, atol=1e-12)
    assert vs[:, 0].max() > 0.1


def test_steady_state_and_isi_closed_form():
    p = wl.NeuronParams(tau_m=10.0, C_m=250.0, I_e=600.0, V_th=20.0, V_reset=10.0, t_ref=2.0)
    net = _one_neuron_net(p)
    sim = on.Simulator(net, np.array([0, 0]), np.zeros(0, np.int64), np.zeros(0, np.int64),
                       np.zeros(0), 8)
    spikes, vs = sim.run(3000, record_v=True)
    v_inf = p.I_e * p.tau_m / p.C_m             # 24 mV > V_th
    h = net.dt
    # first spike: first n with V_inf (1 - e^{-n h / tau_m}) >= V_th
    n1 = next(n for n in range(1, 10000) if v_inf * (1 - math.exp(-n * h / p.tau_m)) >= p.V_th)
    assert spikes[0][0] == n1 - 1               # step index n1-1 completes n1 integrations
    k = next(n for n in range(1, 10000)
             if v_inf + (p.V_reset - v_inf) * math.exp(-n * h / p.tau_m) >= p.V_th)
    isi = np.diff([s for s, _ in spikes])
    assert np.all(isi == 20 + k)
    # sub-threshold steady state
    p2 = wl.NeuronParams(I_e=300.0, V_th=1e9)
    sim2 = on.Simulator(_one_neuron_net(p2), np.array([0, 0]), np.zeros(0, np.int64),
                        np.zeros(0, np.int64), np.zeros(0), 8)
    _, vs2 = sim2.run(2000, record_v=True)
    n = np.arange(1, 2001)
    ref = 300.0 * 10.0 / 250.0 * (1 - np.exp(-n * h / 10.0))
    np.testing.assert_allclose(vs2[:, 0], ref, rtol=0, atol=1e-12)


def test_tau_syn_equal_tau_m_limit():
    h = 0.1
    a = on.propagators(wl.NeuronParams(tau_m=10.0, tau_syn_ex=10.0, tau_syn_in=10.0), h)
    b = on.propagators(wl.NeuronParams(tau_m=10.0, tau_syn_ex=10.0 * (1 + 1e-9),
                                       tau_syn_in=10.0 * (1 + 1e-9)), h)
    assert abs(a["P21_ex"] - b["P21_ex"]) < 1e-12 * a["P21_ex"] * 1e3
    # closed form of the limit: (h / C_m) e^{-h/tau_m}
    assert abs(a["P21_ex"] - h / 250.0 * math.exp(-h / 10.0)) < 1e-18


def test_refractory_clamp():
    p = wl.NeuronParams(I_e=2000.0, t_ref=2.0)
    net = _one_neuron_net(p)
    sim = on.Simulator(net, np.array([0, 0]), np.zeros(0, np.int64), np.zeros(0, np.int64),
                       np.zeros(0), 8)
    spikes, vs = sim.run(200, record_v=True)
    s0 = spikes[0][0]
    assert np.all(vs[s0:s0 + 21, 0] == p.V_reset)       # spike step + 20 refractory steps
    assert vs[s0 + 21, 0] > p.V_reset


def test_delivery_slot_and_receptor():
    net = wl.Network("two", [wl.Population(2, wl.NeuronParams(V_th=1e9))], [], [])
    rp = np.array([0, 2, 2])
    tgt = np.array([1, 1])
    d = np.array([3, 5])
    w = np.array([10.0, -4.0])
    sim = on.Simulator(net, rp, tgt, d, w, 8)
    sim.step_no = 6
    sim.deliver(6, [0])
    assert sim.ring[(6 + 3) % 8, 0, 1] == 10.0
    assert sim.ring[(6 + 5) % 8, 1, 1] == -4.0
    assert np.count_nonzero(sim.ring) == 2


def test_stored_fp32_propagators_round_once():
    p = wl.BALANCED_PARAMS
    net = _one_neuron_net(p)
    a = on.Simulator(net, np.array([0, 0]), np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0), 8)
    b = on.Simulator(net, np.array([0, 0]), np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0), 8,
                     stored_fp32=True)
    for k in ["P22", "P20", "P11_ex", "P21_ex"]:
        assert b.c[k][0] == float(np.float32(a.c[k][0]))
        assert abs(b.c[k][0] - a.c[k][0]) <= 2 ** -24 * abs(a.c[k][0])


def test_poisson_drive_counts_distribution_and_independence():
    """Drive counts (four neurons per Philox block): the count histogram over 40,000
    neuron-steps matches Poisson(nu h) by chi-square, and neighbours that share a block
    (g, g + 1 with g mod 4 = 0) are uncorrelated, as are blocks of consecutive steps."""
    from scipy import stats
    from oracle import sampling as sm
    lam = 20000.0 * 0.1e-3
    thr = sm.poisson_table(20000.0, 0.1)
    n_neurons, steps = 4000, 10
    counts = np.stack([on.poisson_counts(thr, 0, 1234, 0, n_neurons, n) for n in range(steps)])
    flat = counts.ravel()
    assert abs(flat.mean() - lam) < 4 * math.sqrt(lam / flat.size)
    kmax = 7
    obs = np.array([np.count_nonzero(flat == k) for k in range(kmax)] + [np.count_nonzero(flat >= kmax)])
    p = np.array([stats.poisson.pmf(k, lam) for k in range(kmax)] + [stats.poisson.sf(kmax - 1, lam)])
    chi2 = float(np.sum((obs - flat.size * p) ** 2 / (flat.size * p)))
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-3
    for lane in (1, 2, 3):                      # words of one block
        r = np.corrcoef(counts[:, 0::4].ravel(), counts[:, lane::4].ravel())[0, 1]
        assert abs(r) < 4 / math.sqrt(counts[:, 0::4].size)
    r = np.corrcoef(counts[:-1].ravel(), counts[1:].ravel())[0, 1]   # step n vs n + 1
    assert abs(r) < 4 / math.sqrt(counts[:-1].size)
    # a drive over a sub-range draws the same counts as over the whole range
    np.testing.assert_array_equal(on.poisson_counts(thr, 0, 1234, 1001, 57, 3), counts[3, 1001:1058])


def _vinit_net(pops):
    return wl.Network("vinit", [wl.Population(n, p) for n, p in pops], [], [])


def test_initial_v_range_and_uniformity():
    """V0 = lo + (hi - lo) u01(word) lies strictly inside (lo, hi) and is uniform there:
    KS test against U(lo, hi) over 10^5 neurons, per population, with the two
    populations' draws uncorrelated and consecutive neurons uncorrelated."""
    from scipy import stats
    pa = wl.NeuronParams(V_init_lo=-3.0, V_init_hi=19.5, v_init_seed=9)
    pb = wl.NeuronParams(V_init_lo=2.0, V_init_hi=7.0, v_init_seed=9)
    n = 100_000
    v = on.initial_v(_vinit_net([(n, pa), (n, pb)]))
    assert v.shape == (2 * n,)
    for (lo, hi), part in (((-3.0, 19.5), v[:n]), ((2.0, 7.0), v[n:])):
        assert part.min() > lo and part.max() < hi
        assert stats.kstest(part, stats.uniform(loc=lo, scale=hi - lo).cdf).pvalue > 1e-3
    ua = (v[:n] + 3.0) / 22.5
    ub = (v[n:] - 2.0) / 5.0
    lim = 4 / math.sqrt(n)
    assert abs(np.corrcoef(ua, ub)[0, 1]) < lim          # same seed, other population
    assert abs(np.corrcoef(ua[:-1], ua[1:])[0, 1]) < lim  # neighbours


def test_initial_v_exact_at_word_extremes(monkeypatch):
    """The exact V0 for VINIT words 0, 2^9 and 0xFFFFFFFF: u01 gives 2^-24, 3 * 2^-24 and
    1 - 2^-24, so V0 = lo + (hi - lo) u exactly.  The three other words of the block are
    set to other values, so the test also fixes which word is used; the recorded call
    fixes the stream: counter = gid, word2 = population index, purpose VINIT, the
    population's seed."""
    from oracle import philox as ph
    calls = []
    words = np.array([0, 512, 0xFFFFFFFF], dtype=np.uint64)

    def fake_stream(counter, word2, purpose, seed):
        calls.append((np.array(counter), word2, purpose, seed))
        other = np.full(len(counter), 0x80000000, dtype=np.uint64)
        return words[:len(counter)], other, other, other

    monkeypatch.setattr(on.ph, "stream", fake_stream)
    lo, hi = 1.25, 17.75
    p0 = wl.NeuronParams()                                   # lo == hi: no draw
    p1 = wl.NeuronParams(V_init_lo=lo, V_init_hi=hi, v_init_seed=77)
    v = on.initial_v(_vinit_net([(4, p0), (3, p1)]))
    u = np.array([2.0 ** -24, 3 * 2.0 ** -24, 1 - 2.0 ** -24])
    np.testing.assert_array_equal(v[:4], 0.0)
    np.testing.assert_array_equal(v[4:], lo + (hi - lo) * u)
    assert len(calls) == 1
    ctr, word2, purpose, seed = calls[0]
    np.testing.assert_array_equal(ctr, [4, 5, 6])
    assert (word2, purpose, seed) == (1, ph.PURPOSE_VINIT, 77)


def test_initial_v_constant_when_range_is_empty():
    p = wl.NeuronParams(V_init_lo=5.0, V_init_hi=5.0, v_init_seed=1)
    q = wl.NeuronParams(V_init_lo=5.0, V_init_hi=4.0, v_init_seed=1)
    v = on.initial_v(_vinit_net([(10, p), (6, q)]))
    np.testing.assert_array_equal(v, 5.0)
