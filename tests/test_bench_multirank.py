"""bench.py on the CPU: its multi-rank aggregation (N independent replicas, weak
scaling) with two gloo ranks -- units add up, the time is the slowest rank's -- and its
table of measured DRAM traffic per kernel."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist            # noqa: E402
import torch.multiprocessing as mp          # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, ms = bench.aggregate(1000.0 * (rank + 1), 10.0 + 5.0 * rank, dist, "cpu")
    q.put((rank, units, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for _, units, ms in out:
        assert units == 3000.0 and ms == 15.0
    # whole-job throughput = all units over the slowest rank
    assert 3000.0 / (15.0 / 1000.0) == 200000.0


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate(5.0, 2.0) == (5.0, 2.0)


def test_traffic_table_names_existing_kernels():
    """Every kernel of the bench's measured-traffic table is defined in its source file,
    and a figure is reported exactly when that file is unchanged since the capture."""
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for name, d in bench.TRAFFIC.items():
        src = os.path.join(root, "paper_2512_09502_gb300", "csrc", d["source"])
        text = open(src).read()
        kernel = {"finalize_kernel": "finalize_one_rank_kernel"}.get(name, name)
        assert "__global__" in text and (" " + kernel + "(") in text, name
        t = bench.traffic_of(name, 1.0)
        assert (t == d["bytes_per_unit"]) == (bench.file_sha(src) == d["file_sha"]), name
    for name, d in bench.INSTR.items():           # instruction counts: the same rule
        src = os.path.join(root, "paper_2512_09502_gb300", "csrc", d["source"])
        kernel = {"finalize_kernel": "finalize_one_rank_kernel"}.get(name, name)
        assert (" " + kernel + "(") in open(src).read(), name
        assert (bench.inst_of(name) == d["per_unit"]) == (bench.file_sha(src) == d["file_sha"]), name
        assert bench.inst_of(name, "multi_area") is None


def test_reference_arm_json_line():
    """`bench.py --impl reference` times the oracle on a bounded sample and prints one JSON
    line carrying the contract's keys: the arm, the metric and unit of the GPU arm, a value,
    a cpu_baseline describing the sample, and an e2e entry without host-device bytes."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--ref-neurons", "200", "--ref-sim-steps", "50"],
                         capture_output=True, text=True, check=True, timeout=600, cwd=root).stdout
    lines = [x for x in out.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "(synapses + events)/s" and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "200 neurons" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
