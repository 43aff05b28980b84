"""Dry run (Results, "Collective communication: scalable balanced network"): one rank
builds its regular share of a larger network in the absence of the rest.  Its
connections, image rows and R/L maps must be exactly those of that rank in a full build
and in the oracle's per-rank construction."""
import numpy as np
import pytest

from gpu_helpers import compare_rank, ensure_lib, gpu_build, oracle_layout
from paper_2512_09502_gb300 import _lib
from paper_2512_09502_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_lib()


@pytest.mark.parametrize("R,r", [(2, 1), (7, 3), (7, 0), (7, 6)])
def test_dry_run_rank_matches_full_build_and_oracle(R, r):
    net = wl.balanced(240, 61, 30, 8, wl.DELAY_NORMAL, seed=3, n_ranks=R)
    full = gpu_build(net)
    dry = gpu_build(net, dry_run_rank=r)
    _, ref = oracle_layout(net)
    got = dry.get_connections(r)
    compare_rank(got, ref["ranks"][r])
    want = full.get_connections(r)
    for k in ("row_ptr", "tgt", "w", "d"):
        np.testing.assert_array_equal(got[k], want[k])
    for sig in range(R):
        if sig == r:
            continue
        for which in ("R", "L"):
            np.testing.assert_array_equal(dry.get_maps(r, sig, which), full.get_maps(r, sig, which))
            np.testing.assert_array_equal(dry.get_maps(r, sig, which), ref["ranks"][r][which][sig])
    s_dry, s_full = dry.stats(), full.stats()
    assert s_dry["n_synapses"] == len(want["tgt"])
    assert s_dry["n_images"] == len(got["row_ptr"]) - 1 - sum(1 for g in range(net.n_neurons) if g % R == r)
    assert s_dry["peak_device_bytes"] < s_full["peak_device_bytes"]


def test_dry_run_refuses_what_it_did_not_build():
    net = wl.balanced(240, 61, 30, 8, wl.DELAY_NORMAL, seed=3, n_ranks=4)
    dry = gpu_build(net, dry_run_rank=2)
    for call in (lambda: dry.simulate(10), lambda: dry.get_connections(1), lambda: dry.get_maps(2, 0, "S"),
                 lambda: dry.get_maps(0, 2, "R"), lambda: dry.get_spikes()):
        with pytest.raises(_lib.SnnError) as e:
            call()
        assert e.value.code == _lib.SNN_ESTATE


def test_dry_run_of_a_1024_rank_network():
    """Rank 5's share of a balanced network of 1,024 x 20,000 neurons (K = 400 + 100):
    exactly M x K synapses, built without the other 1,023 ranks' connections.  Its
    records carry generation positions (24 bits) where the network-wide counter would
    need 34 bits beside a 31-bit key."""
    R = 1024
    net = wl.balanced(16000 * R, 4000 * R, 400, 100, wl.DELAY_NORMAL, seed=11, n_ranks=R)
    dry = gpu_build(net, dry_run_rank=5)
    s = dry.stats()
    M = sum(1 for _ in range(5, net.n_neurons, R))
    assert s["n_synapses"] == M * 500
    assert s["key_bits"] == 31
    row = dry.get_row(5, 7)                      # local row 7: the outgoing synapses of gid 7 * R + 5
    c = dry.get_connections(5)
    assert c["row_ptr"][-1] == M * 500
    assert (c["tgt"] < M).all() and (c["d"] >= 1).all()
    assert np.array_equal(row[0], c["tgt"][c["row_ptr"][7]:c["row_ptr"][8]])
    assert s["n_images"] > 0 and s["peak_device_bytes"] < 4 << 30
