"""Network-level validation by spiking statistics (the paper's protocol, Methods
"Validation of spiking statistics" and its appendix): three sets of simulations with
different seeds -- two from the oracle, one from the GPU path -- of the 5,000-neuron
balanced network over 1 s.  Per population and statistic (firing rate, CV ISI, pairwise
Pearson correlation of 200 neurons) the Earth Mover's Distance between oracle and GPU
runs must be of the size of the one between two oracle runs with different seeds:
the GPU path adds no variability of its own."""
import numpy as np
import pytest

from gpu_helpers import ensure_lib, gpu_build, oracle_layout
from oracle import connect as oc
from oracle import neuron as on
from paper_2512_09502_gb300 import stats as st
from paper_2512_09502_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

STEPS = 10000            # 1 s of model time at 0.1 ms
T0, T1 = 200.0, 1000.0   # analysis window (ms): the synchronous onset from V = 0 is left out
SEEDS_A, SEEDS_B, SEEDS_GPU = (101, 102, 103), (201, 202, 203), (301, 302, 303)


def _oracle_run(seed):
    net = wl.balanced_small(seed=seed)
    _, ref = oracle_layout(net)
    r = ref["ranks"][0]
    sim = on.Simulator(net, r["row_ptr"], r["tgt"], r["d"], r["w"].astype(np.float32).astype(np.float64),
                       on.ring_slots_for(oc.max_delay(net)), stored_fp32=True)
    spikes, _ = sim.run(STEPS)
    s = np.array([x for x, _ in spikes]), np.array([g for _, g in spikes])
    return st.spike_statistics(*s, st.populations_of(net), net.dt, T0, T1)


def _gpu_run(seed):
    net = wl.balanced_small(seed=seed)
    ctx = gpu_build(net, spike_log_capacity=1 << 22)
    ctx.simulate(STEPS)
    step, gid = ctx.get_spikes()
    ctx.destroy()
    return st.spike_statistics(step, gid, st.populations_of(net), net.dt, T0, T1)


@pytest.fixture(scope="module")
def sets():
    ensure_lib()
    return ([_oracle_run(s) for s in SEEDS_A], [_oracle_run(s) for s in SEEDS_B],
            [_gpu_run(s) for s in SEEDS_GPU])


def test_statistics_emd_gpu_vs_oracle_within_seed_variability(sets):
    a, b, g = sets
    seed_var = st.pairwise_emd(a, b)
    code_var = st.pairwise_emd(a, g)
    rows = []
    for key in sorted(seed_var):
        s_med, c_med = float(np.median(seed_var[key])), float(np.median(code_var[key]))
        rows.append((key, s_med, c_med))
        print(f"{key[0]:>2s} {key[1]:>7s}  EMD seed vs seed {s_med:.4g}  oracle vs GPU {c_med:.4g}")
    for (pop, stat), s_med, c_med in rows:
        assert c_med <= 2.0 * max(seed_var[(pop, stat)]) + 1e-3, (pop, stat, s_med, c_med)
    # the runs are in the paper's regime: asynchronous, irregular, ~8 Hz
    for run in g:
        for pop in ("E", "I"):
            assert 4.0 < run[pop]["rate"].mean() < 16.0
            assert 0.5 < np.median(run[pop]["cv_isi"]) < 1.5
