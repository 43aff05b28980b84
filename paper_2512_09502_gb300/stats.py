"""Spike-train statistics for validating network dynamics (host side).

The paper validates its construction method on the statistics of the spiking activity
rather than on spike trains (Methods, "Validation of spiking statistics"; Appendix,
validation of spike statistics): per population, the distributions of the
time-averaged firing rate of each neuron, of the coefficient of variation of its
inter-spike intervals (CV ISI), and of the pairwise Pearson correlation of binned spike
trains of a subset of 200 neurons.  Two implementations agree when the Earth Mover's
Distance (first-order Wasserstein distance) between their distributions is of the size
of the one between runs of the same implementation with different seeds.

These functions take a recorded spike list ((step, gid) pairs, as returned by
``Context.get_spikes``) and population ranges; they are plain numpy / scipy.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np
from scipy import stats as _st

STATS = ("rate", "cv_isi", "corr")


def spike_statistics(step: np.ndarray, gid: np.ndarray, populations: Sequence[Tuple[str, int, int]],
                     dt_ms: float, t_start_ms: float, t_stop_ms: float, n_corr: int = 200,
                     bin_ms: float = 5.0, subset_seed: int = 0) -> Dict[str, Dict[str, np.ndarray]]:
    """Per population (name, first gid, count): firing rate of every neuron (Hz) over
    [t_start, t_stop); CV ISI of every neuron with at least two intervals there; and the
    Pearson correlation of every pair of a fixed random subset of ``n_corr`` neurons,
    spike counts binned at ``bin_ms`` (silent neurons of the subset are left out)."""
    step = np.asarray(step, dtype=np.int64)
    gid = np.asarray(gid, dtype=np.int64)
    t = step * dt_ms
    keep = (t >= t_start_ms) & (t < t_stop_ms)
    t, gid = t[keep], gid[keep]
    order = np.lexsort((t, gid))
    t, gid = t[order], gid[order]
    dur_s = (t_stop_ms - t_start_ms) / 1000.0
    n_bins = int(np.ceil((t_stop_ms - t_start_ms) / bin_ms))
    out: Dict[str, Dict[str, np.ndarray]] = {}
    rng = np.random.default_rng(subset_seed)
    for name, first, n in populations:
        sel = (gid >= first) & (gid < first + n)
        pg, pt = gid[sel] - first, t[sel]
        counts = np.bincount(pg, minlength=n)
        rate = counts / dur_s
        # CV ISI: spikes are sorted by (neuron, time), so intervals inside a neuron are diffs
        bounds = np.concatenate([[0], np.cumsum(counts)])
        cvs = []
        for k in np.nonzero(counts >= 3)[0]:
            isi = np.diff(pt[bounds[k]:bounds[k + 1]])
            m = isi.mean()
            if m > 0:
                cvs.append(isi.std() / m)
        # pairwise correlation of binned counts of a random subset
        sub = np.sort(rng.choice(n, size=min(n_corr, n), replace=False))
        b = np.minimum(((pt - t_start_ms) / bin_ms).astype(np.int64), n_bins - 1)
        mat = np.zeros((len(sub), n_bins))
        pos = np.searchsorted(sub, pg)
        hit = (pos < len(sub)) & (sub[np.minimum(pos, len(sub) - 1)] == pg)
        np.add.at(mat, (pos[hit], b[hit]), 1.0)
        active = mat.std(axis=1) > 0
        corr = np.array([])
        if active.sum() >= 2:
            cc = np.corrcoef(mat[active])
            corr = cc[np.triu_indices(cc.shape[0], k=1)]
        out[name] = {"rate": rate, "cv_isi": np.array(cvs), "corr": corr}
    return out


def emd(a: np.ndarray, b: np.ndarray) -> float:
    """Earth Mover's Distance between two empirical distributions (1-Wasserstein)."""
    if len(a) == 0 or len(b) == 0:
        return float("nan")
    return float(_st.wasserstein_distance(a, b))


def pairwise_emd(set_a: List[Dict[str, Dict[str, np.ndarray]]], set_b: List[Dict[str, Dict[str, np.ndarray]]]
                 ) -> Dict[Tuple[str, str], List[float]]:
    """EMD of run i of set a against run i of set b, for every population and statistic
    (the paper's pairwise comparison of two sets of simulations)."""
    res: Dict[Tuple[str, str], List[float]] = {}
    for ra, rb in zip(set_a, set_b):
        for pop in ra:
            for s in STATS:
                res.setdefault((pop, s), []).append(emd(ra[pop][s], rb[pop][s]))
    return res


def populations_of(net) -> List[Tuple[str, int, int]]:
    """(name, first gid, count) of a workload's populations, in creation order."""
    out, first = [], 0
    for k, p in enumerate(net.populations):
        out.append((p.name or f"pop{k}", first, p.n))
        first += p.n
    return out


def summarize(res: Dict[Tuple[str, str], List[float]]) -> Dict[str, Dict[str, float]]:
    return {f"{pop}/{s}": {"median": float(np.nanmedian(v)), "max": float(np.nanmax(v))}
            for (pop, s), v in res.items()}


__all__ = ("spike_statistics", "emd", "pairwise_emd", "populations_of", "summarize", "STATS")
