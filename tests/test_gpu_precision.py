"""Stored-weight precision (FP32 / BF16 / FP16 with a power-of-two scale) against the
FP64 oracle with exact (unrounded) weights: membrane error over 100 steps of identical
input, and the first step at which a threshold decision differs.

The network has the in-degrees, weights and delays of the 500k-neuron workload at
5,000 neurons (56M synapses: the size the oracle builds in seconds); V0 is spread up to
threshold so that recurrent spikes flow from the first steps."""
import json

import numpy as np
import pytest

from gpu_helpers import ensure_lib, gpu_build, oracle_layout
from oracle import connect as oc
from oracle import neuron as on
from paper_2512_09502_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

BOUNDS_MV = {"f32": 1e-4, "f16": 2e-2, "bf16": 1e-1}


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_lib()


@pytest.fixture(scope="module")
def reference():
    p = wl.NeuronParams(V_init_lo=0.0, V_init_hi=19.5, v_init_seed=9)
    net = wl.balanced(4000, 1000, 9000, 2250, wl.DELAY_NORMAL, params=p, drive_rate_hz=20000.0)
    syn, ref = oracle_layout(net)
    rk = ref["ranks"][0]
    sim = on.Simulator(net, rk["row_ptr"], rk["tgt"], rk["d"], rk["w"], on.ring_slots_for(oc.max_delay(net)))
    vs, spikes = [], []
    for _ in range(100):
        spikes.append(set(sim.step().tolist()))
        vs.append(sim.V.copy())
    return net, vs, spikes


@pytest.mark.parametrize("fmt", ["f32", "f16", "bf16"])
def test_weight_format_error_vs_fp64(reference, fmt):
    net, vs, spikes = reference
    ctx = gpu_build(net, weight_format=fmt, spike_log_capacity=1 << 22, use_graph=False)
    worst, first_flip = 0.0, None
    for step in range(100):
        ctx.simulate(1)
        st, gid = ctx.get_spikes()
        got = set(gid[st == step].tolist())
        if got != spikes[step]:
            first_flip = step
            break
        V, _, _ = ctx.get_state(0, net.n_neurons)
        worst = max(worst, float(np.max(np.abs(V - vs[step]))))
    n_spk = sum(len(s) for s in spikes[:first_flip if first_flip is not None else 100])
    print("PRECISION", json.dumps({"format": fmt, "max_abs_dV_mV": worst, "first_differing_step": first_flip,
                                   "spikes_compared": n_spk}))
    assert n_spk > 100                     # recurrent input did flow
    assert worst <= BOUNDS_MV[fmt], (fmt, worst)
    if fmt == "f32":
        assert first_flip is None or first_flip > 50
