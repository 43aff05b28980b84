#!/usr/bin/env python3
"""Benchmark of on-device network construction + spike delivery on one GB300.

One step = one pass of the whole hot path over one synthetic network: construction
(counter-based generation of every synapse, the source/delay radix sort, the CSR
layout -- ``snn_calibrate``) followed by ``--sim-steps`` simulation steps (neuron
update + ring-buffer delivery -- ``snn_simulate``), all through the C ABI.

Workload (default): the scaled balanced network, 400k E + 100k I iaf_psc_exp neurons,
fixed in-degree 9,000 E + 2,250 I (5.625G synapses, 50.6 GB layout), delays
normal(1.5, 0.75) ms clipped at 0.1 ms, Poisson drive tuned so that the network fires
at about 8 Hz, 10,000 steps of 0.1 ms.  The metric counts synapses built plus synaptic
events delivered per second of the step.

``--impl reference`` times the CPU oracle (``oracle/``) on a bounded sample of the
same workload instead.  Under torchrun each rank builds and simulates its own replica
(weak scaling; the path needs no exchange between GPUs).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "synapses built/s + synaptic events/s (1 GB300, % HBM peak), bf16 vs fp32 weights"
UNIT = "(synapses + events)/s"
# algorithmic bytes per unit of the measured kernels
BYTES = {"sort_pass": 16.0, "deliver_f32": 13.0, "deliver_bf16": 11.0, "finalize": 17.0, "generate": 8.0,
         "update": 38.0, "update_merged": 30.0}   # update: V, I_ex, I_in, refr r/w, pop r, ring r + clear;
                                                  # merged ring (tau_ex == tau_in): no I_in traffic


WORKLOADS = ("balanced_500k", "balanced_5k", "multi_area", "multi_area_r128", "indegree_x2", "indegree_x5",
             "indegree_x10", "update_500k", "construction_112m", "deliver_500k")


def workload(name: str, scale: float):
    from paper_2512_09502_gb300 import workloads as wl
    # small cases for kernel profiles (a few GB on the device at most, larger than L2)
    if name == "update_500k":           # the full-size neuron update on a layout of a few hundred MB
        p = wl.NeuronParams(V_init_lo=0.0, V_init_hi=19.9, v_init_seed=5)
        return wl.balanced(400000, 100000, 8, 2, wl.DELAY_NORMAL, seed=7, params=p, drive_rate_hz=20000.0,
                           name="update_500k")
    if name == "construction_112m":     # 112.5M synapses, the 500k network's 19-bit source key
        return wl.balanced(240000, 60000, 300, 75, wl.DELAY_NORMAL, seed=7, drive_rate_hz=20000.0,
                           name="construction_112m")
    if name == "deliver_500k":          # the full-size 128 MB ring, 450M synapses, input K x J as at full size
        return wl.balanced(400000, 100000, 720, 180, wl.DELAY_NORMAL, seed=7, drive_rate_hz=20000.0,
                           j_scale=12.5, name="deliver_500k")
    if name == "balanced_500k":
        return wl.balanced_scaled(scale)
    if name == "balanced_5k":
        return wl.balanced_small()
    if name == "multi_area":            # 32 areas, ~1M neurons, 2,328 blocks, one rank
        return wl.multi_area(scale=scale)
    if name == "multi_area_r128":       # the same network over 128 logical ranks
        return wl.multi_area(scale=scale, n_ranks=128)
    if name.startswith("indegree_x"):    # 5.625G synapses with K = 11,250 x factor
        return wl.indegree_scaling(int(name[len("indegree_x"):]), neurons_at_1=int(500_000 * scale))
    raise SystemExit(f"unknown workload {name}")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# DRAM bytes per unit: dram__bytes_read.sum + dram__bytes_write.sum of a one-pass ncu
# capture of the timed step at full size (--cache-control none), divided by the units
# the captured launch processed, with the source file that was measured (sha256[:16] of
# the whole file and the headers it includes at capture time, so that a change anywhere
# in them, inlined helpers included, retires the figure).
TRAFFIC = {
    "gen_kernel": {"bytes_per_unit": 8.00, "source": "build.cu", "file_sha": "9939307653317d86"},
    "onesweep_pass": {"bytes_per_unit": 16.55, "source": "build.cu", "file_sha": "9939307653317d86"},
    "finalize_kernel": {"bytes_per_unit": 17.19, "source": "build.cu", "file_sha": "9939307653317d86"},
    # steady-state steps 2,000+ of the 500k network, direct-load form (the staged form reads
    # the same bytes); per event of the run's average, per neuron
    "deliver_kernel": {"bytes_per_unit": 11.7, "source": "sim.cu", "file_sha": "2bc0cee4c0c0c377"},
    "update_kernel": {"bytes_per_unit": 10.2, "source": "sim.cu", "file_sha": "2bc0cee4c0c0c377"},
}


# the library headers each measured translation unit includes (their inline code is part
# of its kernels)
HEADERS = {"build.cu": ["snn_internal.cuh"], "sim.cu": ["sim_internal.cuh", "snn_internal.cuh"]}


def file_sha(path: str) -> str:
    """sha256[:16] of a source file followed by the library headers it includes."""
    h = hashlib.sha256(open(path, "rb").read())
    for name in HEADERS.get(os.path.basename(path), []):
        h.update(open(os.path.join(os.path.dirname(path), name), "rb").read())
    return h.hexdigest()[:16]


TRAFFIC_WORKLOAD = "balanced_500k"     # the workload the traffic figures were captured on

# Instructions per unit (warp instructions x 32 per record): smsp__inst_executed.sum of a
# capture of each construction kernel on the 112.5M-synapse balanced case, whose 25-bit
# (source, delay) key takes the same digit plan (8, 8, 9 bits) as the 500k network; keyed
# like TRAFFIC.  These kernels are bound by instruction issue, so the bench also reports
# them against the issue ceiling: SMs x 4 schedulers x 32 lanes x the maximum SM clock.
INSTR = {
    "gen_kernel": {"per_unit": 155.0, "source": "build.cu", "file_sha": "9939307653317d86"},
    # at 5.625G records every digit lies in the records' high word: the high-word form's
    # counts (129.5 per 8-bit pass, 147.1 for the 9-bit one)
    "onesweep_pass": {"per_unit": (129.5 + 129.5 + 147.1) / 3, "source": "build.cu", "file_sha": "9939307653317d86"},
    "finalize_kernel": {"per_unit": 231.5, "source": "build.cu", "file_sha": "9939307653317d86"},
}


def inst_of(kernel: str, workload: str = TRAFFIC_WORKLOAD):
    """Measured instructions per unit, when taken on the current source and this workload."""
    d = INSTR.get(kernel)
    if not d or workload != TRAFFIC_WORKLOAD:
        return None
    src = os.path.join(ROOT, "paper_2512_09502_gb300", "csrc", d["source"])
    return d["per_unit"] if file_sha(src) == d["file_sha"] else None


def issue_peak(device: int) -> float:
    """Thread instructions per second at full issue: SMs x 4 schedulers x 32 lanes x the
    maximum SM clock (MEASURED_PEAKS.json, else 2,070 MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        mhz = float(json.load(open(p)).get("sm_max_mhz", mhz))
    return sms * 4 * 32 * mhz * 1e6


PROBE_STEPS_PER_LAUNCH = 8   # the delivery ceiling probe issues 8 steps' events per launch ...
PROBE_LAUNCHES = 20          # ... in 20 launches: launch gaps below 1% of the time

def traffic_of(kernel: str, units_per_launch: float, workload: str = TRAFFIC_WORKLOAD):
    """Measured DRAM bytes per launch, when the figure was taken on the current text of
    the kernel's source file and on this workload (bytes per unit differ between
    workloads: the multi-area ring, for one, is far larger than L2); else None."""
    d = TRAFFIC.get(kernel)
    if not d or workload != TRAFFIC_WORKLOAD:
        return None
    src = os.path.join(ROOT, "paper_2512_09502_gb300", "csrc", d["source"])
    if file_sha(src) != d["file_sha"]:
        return None
    return d["bytes_per_unit"] * units_per_launch


def cpu_sample(scale: float, n_neurons: int = 1000, sim_steps: int = 1000, name: str = "balanced_500k"):
    """The oracle on a bounded sample of the workload: the same balanced network
    (same in-degrees, weights, delays, drive, hence the same dynamical regime) at
    ``n_neurons`` neurons, built and then simulated for ``sim_steps`` steps; or, with
    ``name="balanced_5k"``, the whole 5,000-neuron balanced network."""
    import numpy as np
    from oracle import connect as oc, layout as ol, neuron as on
    from paper_2512_09502_gb300 import workloads as wl
    net = wl.balanced_small() if name == "balanced_5k" else wl.balanced_scaled(scale * n_neurons / 500_000)
    t0 = time.perf_counter()
    syn = oc.generate(net)
    rk = ol.build_rank(syn, ol.round_robin(net.n_neurons, 1), 0)
    sim = on.Simulator(net, rk["row_ptr"], rk["tgt"], rk["d"], rk["w"].astype(np.float32).astype(np.float64),
                       on.ring_slots_for(oc.max_delay(net)))
    spikes, _ = sim.run(sim_steps)
    g = np.array([x for _, x in spikes], dtype=np.int64)
    events = int(np.sum(rk["row_ptr"][g + 1] - rk["row_ptr"][g])) if len(g) else 0
    dt = time.perf_counter() - t0
    units = len(syn["src"]) + events
    what = ("the whole 5,000-neuron balanced network" if name == "balanced_5k" else
            f"balanced network with the workload's in-degrees, weights, delays and drive at {net.n_neurons} neurons")
    return units / dt, dict(synapses=len(syn["src"]), events=events, seconds=dt,
                            sample=f"{what} ({len(syn['src'])} synapses), built then simulated {sim_steps} steps "
                                   f"({events} events)")


def _cpu_worker(job):
    """One replica of the sample in a worker process (top level, so that spawned
    workers can import it); job = (scale, n_neurons, sim_steps), or None to import the
    oracle and return (pool warm-up)."""
    if job is None:
        import oracle.layout  # noqa: F401
        import oracle.neuron  # noqa: F401
        return None
    return cpu_sample(*job)[1]


class CpuPool:
    """Worker processes for the oracle on every host core, started with ``spawn`` (a
    forked child of a process that uses CUDA would hang) and warmed up before any timed
    round."""

    def __init__(self, workers: int):
        import multiprocessing as mp
        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers)
        self.pool.map(_cpu_worker, [None] * workers)

    def round(self, scale: float, n_neurons: int, sim_steps: int):
        """One replica of the sample per worker at once: whole-round units per second
        of wall time, and the sample's description."""
        t0 = time.perf_counter()
        infos = self.pool.map(_cpu_worker, [(scale, n_neurons, sim_steps)] * self.workers)
        dt = time.perf_counter() - t0
        units = sum(i["synapses"] + i["events"] for i in infos)
        return units, dt, infos[0]

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_workers():
    return max(1, min(cpu_cores() or 1, 16))


def cpu_baseline(args):
    """The oracle timed on the host cores: one replica of the bounded sample on one core,
    then one replica per core at once (the sample is independent work, so the all-cores
    figure is the replicas' summed units over the wall time of the round), and the whole
    5,000-neuron balanced network on one core."""
    v1, info = cpu_sample(args.scale, args.ref_neurons, args.ref_sim_steps)
    v5k, info5k = cpu_sample(1.0, sim_steps=1000, name="balanced_5k")
    pool = CpuPool(cpu_workers())
    units, dt, _ = pool.round(args.scale, args.ref_neurons, args.ref_sim_steps)
    pool.close()
    full = 5.625e9 / info["synapses"] * info["seconds"]          # construction share scales with synapses
    return {"value": units / dt, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
            "sample": f"{pool.workers} concurrent replicas (one per core) of: {info['sample']}",
            "serial": {"value": v1, "cores": 1, "seconds": info["seconds"]},
            "balanced_5k_full": {"value": v5k, "cores": 1, "seconds": info5k["seconds"], "sample": info5k["sample"]},
            "full_size_serial_s_extrapolated": full}


def aggregate(units: float, ms: float, dist=None, device: str = "cpu"):
    """Whole-job aggregate over ranks: units summed, time = the slowest rank's."""
    if dist is None:
        return units, ms
    import torch
    u = torch.tensor([units], dtype=torch.float64, device=device)
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


# ---------------------------------------------------------------------------
def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    pool = CpuPool(cpu_workers())
    info = None
    for _ in range(args.warmup):
        pool.round(args.scale, args.ref_neurons, args.ref_sim_steps)
    t0 = time.perf_counter()
    units = 0.0
    for _ in range(args.steps):
        u, _, info = pool.round(args.scale, args.ref_neurons, args.ref_sim_steps)
        units += u
    dt = time.perf_counter() - t0
    pool.close()
    value = units / dt
    sample = f"{pool.workers} concurrent replicas (one per core) of: {info['sample']}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.workers, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2512_09502_gb300 import _lib, build
    build.build()
    net = workload(args.workload, args.scale)
    alloc = _lib.TorchAllocator(local)
    stream = torch.cuda.current_stream()

    # launch parameters: tuned once on this workload (outside every timed region)
    from paper_2512_09502_gb300 import autotune
    tuned = autotune.load()
    if args.autotune and (tuned is None or tuned.get("network") != net.name):
        tuned = autotune.tune(net, allocator=alloc, stream=stream.cuda_stream, device=local,
                              sim_steps=min(args.sim_steps, 2000))
    knobs = {k: int(tuned[k]) for k in ("radix_bits", "sort_items", "deliver_ctas_per_sm", "deliver_mode")
             if k in tuned} if tuned else {}
    for k in ("radix_bits", "sort_items", "deliver_ctas_per_sm"):
        if getattr(args, k):
            knobs[k] = getattr(args, k)
    extra = {"xi": args.xi} if args.xi else {}
    if args.deliver_mode is not None:
        knobs["deliver_mode"] = args.deliver_mode

    def one(fmt, sim_steps, profile=False, after=None):
        ctx = _lib.build_network(net, weight_format=fmt, allocator=alloc, stream=stream.cuda_stream,
                                 device=local, use_graph=True, profile_kernels=profile, **knobs, **extra)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.calibrate()
        ctx.simulate(sim_steps)
        e1.record(stream)
        e1.synchronize()
        st = ctx.stats()
        if after is not None:
            after(ctx, st)
        ctx.destroy()
        return e0.elapsed_time(e1), st

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()


    def timed(fmt):
        for _ in range(args.warmup):
            one(fmt, args.sim_steps)
        barrier()
        clk = Clocks(local)
        clk.start()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        torch.cuda.nvtx.range_push(f"timed_{fmt}")     # lets a profiler select the timed steps
        stats = []
        for _ in range(args.steps):
            stats.append(one(fmt, args.sim_steps)[1])
        torch.cuda.nvtx.range_pop()
        t1.record(stream)
        barrier()
        clocks = clk.stop()
        units, ms = aggregate(sum(s["n_synapses"] + s["n_events"] for s in stats), t0.elapsed_time(t1),
                              dist, "cuda")
        return ms, units, stats, clocks

    ms, units, stats, clocks = timed("f32")
    value = units / (ms / 1000.0)
    s0 = stats[-1]
    syn_per_s = s0["n_synapses"] / (s0["t_calibrate_ms"] / 1000.0)
    ev_per_s = s0["n_events"] / (s0["t_simulate_ms"] / 1000.0) if s0["t_simulate_ms"] else 0.0
    launches = sum(s["kernel_launches"] for s in stats)

    # BF16-weight form of the same workload
    bf = None
    if not args.no_bf16:
        ms_b, units_b, stats_b, _ = timed("bf16")
        sb = stats_b[-1]
        bf = {"value": units_b / (ms_b / 1000.0),
              "synapses_built_per_s": sb["n_synapses"] / (sb["t_calibrate_ms"] / 1000.0),
              "synaptic_events_per_s": sb["n_events"] / (sb["t_simulate_ms"] / 1000.0) if sb["t_simulate_ms"] else 0.0}
        bf["events_per_s_vs_f32"] = bf["synaptic_events_per_s"] / ev_per_s if ev_per_s else None

    # end to end through the public API: host spec in, stats (the result) out
    e2e_ms, e2e_units, h2d, d2h = 0.0, 0.0, 0, 0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx = _lib.build_network(net, weight_format="f32", allocator=alloc, stream=stream.cuda_stream,
                                 device=local, use_graph=True, **knobs, **extra)
        ctx.calibrate()
        ctx.simulate(args.sim_steps)
        st = ctx.stats()
        ctx.destroy()
        e2e_ms += 1000 * (time.perf_counter() - t)
        e2e_units += st["n_synapses"] + st["n_events"]
        h2d, d2h = st["h2d_bytes"], st["d2h_bytes"]
    e2e_units, e2e_ms = aggregate(e2e_units, e2e_ms, dist, "cuda")

    # per-kernel CUDA-event times for the roofline (outside the timed region), and the
    # delivery's ceiling: the same ring reductions issued by the probe kernel
    probe = {}

    def run_probe(ctx, st):
        if net.n_ranks != 1 or not args.sim_steps or not st["n_events"]:
            return
        n = int(min(st["n_synapses"], PROBE_STEPS_PER_LAUNCH * st["n_events"] / max(st["steps_done"], 1)))
        for mode in (0, 1):
            ctx.ring_reduction_probe(mode, n, 2)                       # warm-up
            probe[mode] = n / (ctx.ring_reduction_probe(mode, n, PROBE_LAUNCHES) / 1000.0)
        probe["n"] = n

    _, prof = one("f32", min(args.sim_steps, 2000), profile=True, after=run_probe)
    peak, peak_kind = peaks()
    E = prof["n_synapses"]
    step_ms = ms / args.steps
    dl = max(prof["deliver_launches"], 1)
    ev_launch = prof["n_events"] / dl
    kern = {
        "gen_kernel": dict(ms=prof["t_generate_ms"], launches=1, units=E, bpu=BYTES["generate"], bound="alu"),
        "onesweep_pass": dict(ms=prof["t_sort_pass_ms"] / max(prof["sort_passes"], 1), launches=prof["sort_passes"],
                              units=E, bpu=BYTES["sort_pass"], bound="hbm"),
        "finalize_kernel": dict(ms=prof["t_finalize_ms"], launches=1, units=E, bpu=BYTES["finalize"], bound="hbm"),
        "update_kernel": dict(ms=prof["t_update_ms"] / max(prof["update_launches"], 1), launches=args.sim_steps,
                              units=net.n_neurons, bound="hbm",
                              bpu=BYTES["update_merged" if all(p.params.tau_syn_ex == p.params.tau_syn_in
                                                               for p in net.populations) else "update"]),
        "deliver_kernel": dict(ms=prof["t_deliver_ms"] / dl, launches=args.sim_steps, units=ev_launch,
                               bpu=BYTES["deliver_f32"], bound="hbm"),
    }
    # In the timed steps the simulation runs as CUDA graphs, where single kernels are not
    # timed.  On one rank the delivery is the critical path of a step (the neuron work
    # of the step runs beside it on a second stream), so the timed simulation's time per
    # step bounds its in-step duration from above, and the roofline uses that bound.
    # The per-launch time of the profiled run (events around every launch, no graph)
    # is reported beside it; with several ranks (update -> route -> deliver in sequence)
    # the profiled time is the one used.
    sim_per_step = s0["t_simulate_ms"] / max(args.sim_steps, 1)
    kern["deliver_kernel"]["profiled_ms"] = kern["deliver_kernel"]["ms"]
    if args.sim_steps and net.n_ranks == 1:
        kern["deliver_kernel"]["ms"] = sim_per_step
        kern["deliver_kernel"]["units"] = s0["n_events"] / args.sim_steps
    table = {}
    ipk = issue_peak(local)
    for k, v in kern.items():
        gbps = v["units"] * v["bpu"] / (v["ms"] / 1000.0) / 1e9 if v["ms"] else None
        table[k] = {"ms_per_launch": v["ms"], "launches_per_step": v["launches"],
                    "share_of_step": v["ms"] * v["launches"] / step_ms, "algorithmic_GBps": gbps,
                    "frac_of_hbm": gbps / peak if gbps else None,
                    "traffic_bytes_per_launch": traffic_of(k, v["units"], args.workload)}
        ipu = inst_of(k, args.workload)
        if ipu is not None and v["ms"]:
            table[k]["bound"] = "issue"
            table[k]["instructions_per_unit"] = ipu
            table[k]["issue_frac"] = v["units"] * ipu / (v["ms"] / 1000.0) / ipk
    table["deliver_kernel"]["ms_per_launch_profiled"] = kern["deliver_kernel"]["profiled_ms"]
    table["update_kernel"]["timing"] = "profiled run, events around every launch"
    if net.n_ranks == 1:
        table["deliver_kernel"]["timing"] = "timed graph steps: simulation time per step (upper bound of the launch)"
        # the neuron work runs beside the delivery, inside the step time charged to it
        table["update_kernel"]["share_of_step"] = None
        table["update_kernel"]["overlapped_with_deliver_in_timed_step"] = True
    else:
        table["deliver_kernel"]["timing"] = "profiled run, events around every launch"
    dom = max((k for k in kern if kern[k]["bound"] == "hbm" and table[k]["share_of_step"] is not None),
              key=lambda k: table[k]["share_of_step"])
    d = kern[dom]
    alg = d["units"] * d["bpu"]
    ach = alg / (d["ms"] / 1000.0) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_kind": peak_kind, "traffic": traffic_of(dom, d["units"], args.workload),
            "algorithmic_bytes_per_launch": alg,
            "kernels": table}
    if probe and dom == "deliver_kernel":
        dev = d["units"] / (d["ms"] / 1000.0)
        roof["ceiling"] = {
            "what": "the delivery's ring reductions replayed by snn_ring_reduction_probe (adds zeros): "
                    "'streamed' = the direct delivery's loop over consecutive synapses, no spike list; "
                    "'reductions_only' = the same delays with hashed targets, nothing streamed",
            "events_per_launch": probe["n"], "launches": PROBE_LAUNCHES,
            "streamed_events_per_s": probe[0], "reductions_only_events_per_s": probe[1],
            "deliver_events_per_s": dev, "frac_of_streamed": dev / probe[0], "frac_of_reductions_only": dev / probe[1]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "neurons": net.n_neurons, "synapses": s0["n_synapses"],
                       "sim_steps": args.sim_steps, "dt_ms": net.dt, "drive_hz": net.drives[0].rate_hz if net.drives else 0.0,
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "n_ranks": net.n_ranks, "l2": "working set (connection layout) far larger than L2",
                       "deliver_mode": "direct loads" if knobs.get("deliver_mode", 0) else "staged bulk copies"},
            "components": {"synapses_built_per_s": syn_per_s, "synaptic_events_per_s": ev_per_s,
                           "construct_ms": s0["t_calibrate_ms"], "simulate_ms": s0["t_simulate_ms"],
                           "generate_ms": s0["t_generate_ms"], "sort_ms": s0["t_sort_ms"],
                           "finalize_ms": s0["t_finalize_ms"], "events_per_step": s0["n_events"] / max(args.sim_steps, 1),
                           "rate_hz": s0["n_spikes"] / net.n_neurons / (args.sim_steps * net.dt / 1000.0)
                           if args.sim_steps else 0.0,
                           "maps_ms": s0["t_maps_ms"], "n_images": s0["n_images"], "xi": args.xi,
                           "peak_device_GB": s0["peak_device_bytes"] / 1e9},
            "bf16": bf,
            "tuned": knobs,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_units / (e2e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="balanced_500k", choices=WORKLOADS)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--sim-steps", type=int, default=10_000)
    ap.add_argument("--ref-neurons", type=int, default=1000)
    ap.add_argument("--ref-sim-steps", type=int, default=1000)
    ap.add_argument("--no-bf16", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    # launch parameters (override the tuner) and the all-sources image threshold
    ap.add_argument("--radix-bits", dest="radix_bits", type=int, default=0)
    ap.add_argument("--sort-items", dest="sort_items", type=int, default=0)
    ap.add_argument("--deliver-ctas", dest="deliver_ctas_per_sm", type=int, default=0)
    ap.add_argument("--xi", type=float, default=0.0)
    ap.add_argument("--deliver-mode", dest="deliver_mode", type=int, default=None,
                    help="0: staged chunks (bulk copies), 1: direct loads (default: tuned)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
