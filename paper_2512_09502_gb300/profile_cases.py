"""Small cases for kernel profiling (a few GB on the device at most).

    python -m paper_2512_09502_gb300.profile_cases update_500k       # update at 500k neurons
    python -m paper_2512_09502_gb300.profile_cases construction_112m # gen, sort, finalize
    python -m paper_2512_09502_gb300.profile_cases deliver_500k      # delivery, full-size ring

Each builds one network and runs it; a profiler selects the kernel launches it wants.
"""
from __future__ import annotations

import sys


def _ctx(net, **kw):
    from . import _lib
    return _lib.build_network(net, allocator=_lib.TorchAllocator(0), **kw)


def update_500k():
    """500k neurons with in-degree 8 + 2: the full-size neuron update on a layout of a
    few hundred MB (its rate is higher than the 5.625G-synapse workload's)."""
    from . import workloads as wl
    p = wl.NeuronParams(V_init_lo=0.0, V_init_hi=19.9, v_init_seed=5)
    net = wl.balanced(400000, 100000, 8, 2, wl.DELAY_NORMAL, seed=7, params=p, drive_rate_hz=20000.0)
    ctx = _ctx(net, use_graph=False)
    ctx.calibrate()
    ctx.simulate(300)
    s = ctx.stats()
    print("spikes/step", s["n_spikes"] / 300, "events/step", s["n_events"] / 300)


def construction_112m():
    """100k neurons, in-degree 900 + 225: 112.5M synapses (about 1.9 GB at peak)."""
    from . import workloads as wl
    net = wl.balanced(80000, 20000, 900, 225, wl.DELAY_NORMAL, seed=7, drive_rate_hz=20000.0)
    ctx = _ctx(net, radix_bits=9, sort_items=16, deliver_ctas_per_sm=16)
    ctx.calibrate()
    s = ctx.stats()
    print("synapses", s["n_synapses"], "gen", s["t_generate_ms"], "sort", s["t_sort_ms"], "finalize",
          s["t_finalize_ms"])


def deliver_500k():
    """500k neurons with in-degree 720 + 180 and weights x12.5 (the input K x J of the
    5.625G-synapse workload): the full-size 128 MB ring with a 450M-synapse layout."""
    from . import workloads as wl
    net = wl.balanced(400000, 100000, 720, 180, wl.DELAY_NORMAL, seed=7, drive_rate_hz=20000.0, j_scale=12.5)
    ctx = _ctx(net, use_graph=False, radix_bits=9, sort_items=16, deliver_ctas_per_sm=16)
    ctx.calibrate()
    ctx.simulate(400)
    s = ctx.stats()
    print("spikes/step", s["n_spikes"] / 400, "events/step", s["n_events"] / 400)


CASES = {"update_500k": update_500k, "construction_112m": construction_112m, "deliver_500k": deliver_500k}

if __name__ == "__main__":
    if len(sys.argv) != 2 or sys.argv[1] not in CASES:
        raise SystemExit("usage: python -m paper_2512_09502_gb300.profile_cases " + "|".join(CASES))
    CASES[sys.argv[1]]()
