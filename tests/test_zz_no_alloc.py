"""The allocation-free construction entry point (snn_connect_sorted_noalloc) against
the regular path (snn_calibrate + snn_get_connections), through the C ABI.

Callers that cannot call cudaMalloc -- a host application that owns every byte of
device memory under a fixed budget, such as a simulator embedding this library --
pass their own output buffers; the entry point keeps its intermediates in a fixed
device scratch array.  This file is collected last so that a run stopping at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from gpu_helpers import ensure_lib, f32_ulp_distance, gpu_build
from paper_2512_09502_gb300 import _lib, workloads as wl

pytestmark = pytest.mark.gpu


def _projection(kind):
    """One projection of each shape the entry point builds: fixed in-degree with normal
    delays, fixed total number (the draw-indexed generation branch) and a constant
    delay (the branch without a delay table)."""
    p = wl.BALANCED_PARAMS
    w = wl.Dist(wl.W_NORMAL_SIGN, 87.8, 8.78)
    if kind == "fixed_indegree":
        pr = wl.Projection(0, 2500, 0, 3000, wl.Rule(wl.RULE_FIXED_INDEGREE, 50), w, wl.DELAY_NORMAL, 1234)
    elif kind == "fixed_total":
        pr = wl.Projection(500, 2000, 0, 3000, wl.Rule(wl.RULE_FIXED_TOTAL, 150_000), w, wl.DELAY_NORMAL, 77)
    else:
        pr = wl.Projection(0, 3000, 1000, 1700, wl.Rule(wl.RULE_FIXED_INDEGREE, 40), w,
                           wl.Dist(wl.D_CONST, 1.5), 9)
    net = wl.Network("noalloc", [wl.Population(3000, p)], [pr], [])
    return net, pr


def _call(lib, torch, n_neurons, pr, cap, stream):
    rp = torch.zeros(n_neurons + 1, dtype=torch.int64, device="cuda")
    tgt = torch.zeros(cap, dtype=torch.int32, device="cuda")
    w = torch.zeros(cap, dtype=torch.float32, device="cuda")
    d = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    rule = _lib.snn_rule(_lib.RULES[pr.rule.kind], float(pr.rule.param))
    wd = _lib.snn_dist(_lib.W_KINDS[pr.weight.kind], pr.weight.mean, pr.weight.sd, pr.weight.lo)
    dd = _lib.snn_dist(_lib.D_KINDS[pr.delay.kind], pr.delay.mean, pr.delay.sd, pr.delay.lo)
    n = C.c_uint64()
    msg = C.create_string_buffer(256)
    rc = lib.snn_connect_sorted_noalloc(n_neurons, pr.src_first, pr.n_src, pr.tgt_first, pr.n_tgt,
                                        C.byref(rule), C.byref(wd), C.byref(dd), pr.seed, 0.1,
                                        C.c_void_p(rp.data_ptr()), C.c_void_p(tgt.data_ptr()),
                                        C.c_void_p(w.data_ptr()), C.c_void_p(d.data_ptr()), cap,
                                        C.byref(n), C.c_void_p(stream), msg, len(msg))
    return rc, n.value, msg.value.decode(), rp, tgt, w, d


@pytest.mark.parametrize("kind", ["fixed_indegree", "fixed_total", "const_delay"])
def test_noalloc_matches_calibrate_twice(kind):
    torch = pytest.importorskip("torch")
    lib = ensure_lib()
    net, pr = _projection(kind)
    ref_ctx = gpu_build(net)
    ref = ref_ctx.get_connections(0)
    ref_ctx.destroy()
    E = len(ref["tgt"])
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                    # the scratch keeps the previous call's contents
        rc, n, msg, rp, tgt, w, d = _call(lib, torch, net.n_neurons, pr, E, stream)
        assert rc == 0, msg
        assert n == E
        np.testing.assert_array_equal(rp.cpu().numpy(), ref["row_ptr"])
        np.testing.assert_array_equal(tgt.cpu().numpy().view(np.uint32), ref["tgt"])
        np.testing.assert_array_equal(d.cpu().numpy(), ref["d"])
        assert f32_ulp_distance(w.cpu().numpy(), ref["w"]).max() <= 4


def test_noalloc_rejects_sizes_over_the_limit():
    torch = pytest.importorskip("torch")
    lib = ensure_lib()
    n_neurons = 100_000
    pr = wl.Projection(0, n_neurons, 0, n_neurons, wl.Rule(wl.RULE_FIXED_INDEGREE, 20),
                       wl.Dist(wl.W_CONST, 1.0), wl.Dist(wl.D_CONST, 1.0), 1)
    rc, n, msg, *_ = _call(lib, torch, n_neurons, pr, 16, torch.cuda.current_stream().cuda_stream)
    assert rc == -1 and "limit" in msg
