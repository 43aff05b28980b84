"""Spike-statistics helpers (host side) against closed forms and constructed trains."""
import numpy as np

from paper_2512_09502_gb300 import stats as st

DT = 0.1


def _spikes(trains):
    """trains: {gid: spike times in ms} -> (step, gid) arrays on the dt grid."""
    step, gid = [], []
    for g, ts in trains.items():
        step += [int(round(x / DT)) for x in ts]
        gid += [g] * len(ts)
    return np.array(step), np.array(gid)


def test_regular_train_rate_and_zero_cv():
    step, gid = _spikes({0: np.arange(5.0, 1000.0, 10.0), 1: np.arange(5.0, 1000.0, 25.0)})
    s = st.spike_statistics(step, gid, [("P", 0, 2)], DT, 0.0, 1000.0)["P"]
    np.testing.assert_allclose(s["rate"], [100.0, 40.0])
    np.testing.assert_allclose(s["cv_isi"], [0.0, 0.0], atol=1e-9)


def test_poisson_trains_cv_near_one_and_uncorrelated():
    rng = np.random.default_rng(5)
    trains = {g: np.sort(rng.uniform(0, 100000.0, rng.poisson(20 * 100))) for g in range(200)}
    step, gid = _spikes(trains)
    s = st.spike_statistics(step, gid, [("P", 0, 200)], DT, 0.0, 100000.0, n_corr=200, bin_ms=5.0)["P"]
    assert abs(s["rate"].mean() - 20.0) < 0.5
    assert abs(s["cv_isi"].mean() - 1.0) < 0.03          # exponential intervals
    assert len(s["corr"]) == 200 * 199 // 2
    assert abs(s["corr"].mean()) < 0.005


def test_identical_trains_fully_correlated_and_window():
    ts = np.arange(3.0, 2000.0, 17.0)
    step, gid = _spikes({0: ts, 1: ts, 2: ts + 0.0})
    s = st.spike_statistics(step, gid, [("P", 0, 3)], DT, 500.0, 1500.0, n_corr=3, bin_ms=1.0)["P"]
    np.testing.assert_allclose(s["corr"], [1.0, 1.0, 1.0])
    expected = np.count_nonzero((ts >= 500.0) & (ts < 1500.0)) / 1.0
    np.testing.assert_allclose(s["rate"], [expected] * 3)


def test_emd_closed_forms():
    x = np.random.default_rng(1).normal(size=1000)
    assert st.emd(x, x) == 0.0
    assert abs(st.emd(x, x + 0.37) - 0.37) < 1e-12       # a shift moves every unit of mass by 0.37
    assert abs(st.emd(np.zeros(4), np.ones(4)) - 1.0) < 1e-12


def test_pairwise_emd_and_populations():
    from paper_2512_09502_gb300 import workloads as wl
    net = wl.balanced_small()
    pops = st.populations_of(net)
    assert pops == [("E", 0, 4000), ("I", 4000, 1000)]
    rng = np.random.default_rng(2)
    runs = []
    for _ in range(2):
        trains = {g: np.sort(rng.uniform(0, 1000.0, 8)) for g in range(0, 5000, 7)}
        runs.append(st.spike_statistics(*_spikes(trains), pops, DT, 0.0, 1000.0, n_corr=50))
    res = st.pairwise_emd([runs[0]], [runs[1]])
    assert set(res) == {(p, s) for p, _, _ in pops for s in st.STATS}
    assert all(len(v) == 1 and v[0] >= 0 for v in res.values())
