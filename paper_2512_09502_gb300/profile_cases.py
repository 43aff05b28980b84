"""Small cases for kernel profiling (a few GB on the device at most).

    python -m paper_2512_09502_gb300.profile_cases update_500k       # update at 500k neurons
    python -m paper_2512_09502_gb300.profile_cases construction_112m # gen, sort, finalize
    python -m paper_2512_09502_gb300.profile_cases deliver_500k      # delivery, full-size ring
    python -m paper_2512_09502_gb300.profile_cases images_xi_multi_area_r128

The first three build one network and run it; a profiler selects the kernel launches
it wants.  The last measures the all-sources image threshold xi (0 and 1) on the
multi-area network over 128 logical ranks and prints one JSON line per build.
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
    """300k neurons, in-degree 300 + 75: 112.5M synapses (about 2 GB at peak), sorted on
    a 19-bit key like the 500k network's (a 9- and a 10-bit pass)."""
    from . import workloads as wl
    net = wl.balanced(240000, 60000, 300, 75, wl.DELAY_NORMAL, seed=7, drive_rate_hz=20000.0)
    ctx = _ctx(net, radix_bits=10, sort_items=16, deliver_ctas_per_sm=16)
    ctx.calibrate()
    s = ctx.stats()
    print("synapses", s["n_synapses"], "gen", s["t_generate_ms"], "sort", s["t_sort_ms"], "finalize",
          s["t_finalize_ms"])


def deliver_500k():
    """500k neurons with in-degree 720 + 180 and weights x12.5 (the input K x J of the
    5.625G-synapse workload): the full-size 128 MB ring with a 450M-synapse layout."""
    from . import workloads as wl
    net = wl.balanced(400000, 100000, 720, 180, wl.DELAY_NORMAL, seed=7, drive_rate_hz=20000.0, j_scale=12.5)
    ctx = _ctx(net, use_graph=False, radix_bits=10, sort_items=16, deliver_ctas_per_sm=16)
    ctx.calibrate()
    ctx.simulate(400)
    s = ctx.stats()
    print("spikes/step", s["n_spikes"] / 400, "events/step", s["n_events"] / 400)


def images_xi_multi_area_r128():
    """Flagged images (xi = 0) against all-sources images (xi = 1, the paper's value) on
    the 32-area network over 128 ranks: map construction time, images, peak device
    memory, and the simulation of 1,000 steps (images without connections add routed,
    empty rows).  Each setting is built twice; the first build warms the allocator."""
    import json
    from . import workloads as wl
    net = wl.multi_area(seed=1234, n_ranks=128)
    for xi in (0.0, 1.0, 0.0, 1.0):
        ctx = _ctx(net, xi=xi)
        ctx.calibrate()
        ctx.simulate(1000)
        s = ctx.stats()
        print(json.dumps({"xi": xi, "n_synapses": s["n_synapses"], "n_images": s["n_images"],
                          "t_maps_ms": round(s["t_maps_ms"], 2), "t_calibrate_ms": round(s["t_calibrate_ms"], 2),
                          "peak_device_GB": round(s["peak_device_bytes"] / 1e9, 3),
                          "t_simulate_1000_steps_ms": round(s["t_simulate_ms"], 1),
                          "spikes": s["n_spikes"], "events": s["n_events"]}), flush=True)
        ctx.destroy()


CASES = {"update_500k": update_500k, "construction_112m": construction_112m, "deliver_500k": deliver_500k,
         "images_xi_multi_area_r128": images_xi_multi_area_r128}

if __name__ == "__main__":
    if len(sys.argv) != 2 or sys.argv[1] not in CASES:
        raise SystemExit("usage: python -m paper_2512_09502_gb300.profile_cases " + "|".join(CASES))
    CASES[sys.argv[1]]()
