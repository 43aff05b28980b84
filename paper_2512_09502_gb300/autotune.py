"""Autotuner for the library's launch parameters.

Sweeps, on the network it is given (construct + simulate through the C ABI):
  * radix_bits x sort_items  -> construction time (generation + sort + finalize);
  * delivery form x deliver_ctas_per_sm -> simulation time per delivered event (the
    staged form, whose shared memory caps its resident CTAs, and direct loads);
and caches the fastest setting as JSON (``SNN_AUTOTUNE_CACHE`` or
``paper_2512_09502_gb300/_build/autotune.json``).  ``_lib.Context`` applies a cached
setting to every tunable left at 0.
"""
from __future__ import annotations

import json
import os
import time
from typing import Optional

from . import _lib

CACHE = os.environ.get("SNN_AUTOTUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json"))
SORT_SPACE = [(rb, it) for rb in (8, 9, 10) for it in (8, 12, 16)]
# (deliver_mode, deliver_ctas_per_sm): 0 = staged chunks, 1 = direct loads
DELIVER_SPACE = ((0, 1), (0, 2), (0, 4), (1, 4), (1, 8), (1, 16))


def load(path: Optional[str] = None) -> Optional[dict]:
    path = path or CACHE
    if not os.path.exists(path):
        return None
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return None


def tune(net, *, allocator=None, stream=None, device: int = 0, sim_steps: int = 1000,
         repeats: int = 1, path: Optional[str] = None) -> dict:
    """Measure every candidate on ``net`` and write the winner to the cache."""
    t0 = time.time()
    rows = []
    best_sort, best_t = None, float("inf")
    for rb, it in SORT_SPACE:
        ts = []
        for _ in range(repeats):
            ctx = _lib.build_network(net, allocator=allocator, stream=stream, device=device, radix_bits=rb,
                                     sort_items=it, deliver_ctas_per_sm=8)
            ctx.calibrate()
            ts.append(ctx.stats()["t_calibrate_ms"])
            ctx.destroy()
        t = min(ts)
        rows.append({"radix_bits": rb, "sort_items": it, "construct_ms": t})
        if t < best_t:
            best_sort, best_t = (rb, it), t
    best_cps, best_mode, best_ns = None, 0, float("inf")
    for mode, cps in DELIVER_SPACE:
        ctx = _lib.build_network(net, allocator=allocator, stream=stream, device=device, radix_bits=best_sort[0],
                                 sort_items=best_sort[1], deliver_ctas_per_sm=cps, deliver_mode=mode,
                                 use_graph=True)
        ctx.calibrate()
        ctx.simulate(sim_steps)
        st = ctx.stats()
        ctx.destroy()
        ns_per_event = 1e6 * st["t_simulate_ms"] / max(st["n_events"], 1)
        rows.append({"deliver_mode": mode, "deliver_ctas_per_sm": cps, "sim_ns_per_event": ns_per_event})
        if ns_per_event < best_ns:
            best_cps, best_mode, best_ns = cps, mode, ns_per_event
    out = {"radix_bits": best_sort[0], "sort_items": best_sort[1], "deliver_ctas_per_sm": best_cps,
           "deliver_mode": best_mode,
           "network": net.name, "neurons": net.n_neurons, "seconds": time.time() - t0, "measurements": rows}
    path = path or CACHE
    os.makedirs(os.path.dirname(path), exist_ok=True)
    json.dump(out, open(path, "w"), indent=1)
    return out
