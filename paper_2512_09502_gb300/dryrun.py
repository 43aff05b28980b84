"""Dry-run estimation of one rank's share of a large balanced network.

The paper estimates the memory and construction time of configurations larger than
the machine at hand by letting a process build its regular share of the network in the
absence of the rest (Results, "Collective communication: scalable balanced network").
This command does that on one GPU for the balanced network (80% E / 20% I, fixed
in-degree K_E + K_I, weights and delays as in the 500k workload): it builds rank
``--rank`` of an ``--ranks``-rank network with ``--per-rank`` neurons per rank and
prints one JSON line per repetition with the rank's synapse and image counts, the
construction phases' device times and the peak device memory.

    python -m paper_2512_09502_gb300.dryrun --ranks 1024 --per-rank 112500
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--ranks", type=int, default=1024)
    ap.add_argument("--per-rank", type=int, default=112500, help="neurons per rank")
    ap.add_argument("--rank", type=int, default=3)
    ap.add_argument("--k-e", type=int, default=9000)
    ap.add_argument("--k-i", type=int, default=2250)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--xi", type=float, default=0.0, help="all-sources image threshold (0: flagged images)")
    ap.add_argument("--device", type=int, default=0)
    args = ap.parse_args(argv)

    from . import _lib, workloads as wl
    alloc = _lib.TorchAllocator(args.device)
    R, per = args.ranks, args.per_rank
    ne, ni = per * 4 // 5, per - per * 4 // 5
    net = wl.balanced(ne * R, ni * R, args.k_e, args.k_i, wl.DELAY_NORMAL, seed=1234, n_ranks=R,
                      drive_rate_hz=0.0)
    for _ in range(args.repeat):
        t0 = time.perf_counter()
        ctx = _lib.build_network(net, allocator=alloc, device=args.device, dry_run_rank=args.rank,
                                 xi=args.xi)
        t1 = time.perf_counter()
        ctx.calibrate()
        t2 = time.perf_counter()
        s = ctx.stats()
        ctx.destroy()
        print(json.dumps({
            "ranks": R, "rank": args.rank, "xi": args.xi, "neurons_per_rank": per, "network_neurons": net.n_neurons,
            "network_synapses": net.n_neurons * (args.k_e + args.k_i),
            "rank_synapses": s["n_synapses"], "rank_images": s["n_images"],
            "key_bits": s["key_bits"], "sort_passes": s["sort_passes"],
            "t_generate_ms": s["t_generate_ms"], "t_sort_ms": s["t_sort_ms"],
            "t_finalize_ms": s["t_finalize_ms"], "t_maps_ms": s["t_maps_ms"],
            "t_calibrate_ms": s["t_calibrate_ms"], "calibrate_wall_s": t2 - t1, "create_wall_s": t1 - t0,
            "peak_device_GB": s["peak_device_bytes"] / 1e9}), flush=True)


if __name__ == "__main__":
    main()
