"""Shared helpers of the GPU parity tests: build through the C ABI, build with the
oracle, compare."""
import numpy as np

from oracle import connect as oc
from oracle import layout as ol
from paper_2512_09502_gb300 import _lib, build


def ensure_lib():
    build.build()
    return _lib.load()


def gpu_build(net, **kw):
    ctx = _lib.build_network(net, **kw)
    ctx.calibrate()
    return ctx


def oracle_layout(net, R=None, xi=0.0):
    R = net.n_ranks if R is None else R
    syn = oc.generate(net)
    part = ol.round_robin(net.n_neurons, R)
    return syn, ol.build_all(syn, part, ol.forced_images(net, part, xi))


def compare_maps(ctx, ref, R):
    """Every map of every rank pair (R, L, S, T/P, H, I, G/Q) equal to the oracle's."""
    for tau in range(R):
        for sig in range(R):
            if sig == tau:
                continue
            np.testing.assert_array_equal(ctx.get_maps(tau, sig, "R"), ref["ranks"][tau]["R"][sig])
            np.testing.assert_array_equal(ctx.get_maps(tau, sig, "L"), ref["ranks"][tau]["L"][sig])
            np.testing.assert_array_equal(ctx.get_maps(tau, sig, "S"), ref["S"][sig][tau])
    for sig in range(R):
        ptr, T, P = ref["TP"][sig]
        np.testing.assert_array_equal(ctx.get_maps(0, sig, "TP_PTR"), ptr)
        np.testing.assert_array_equal(ctx.get_maps(0, sig, "T"), T)
        np.testing.assert_array_equal(ctx.get_maps(0, sig, "P"), P)
        np.testing.assert_array_equal(ctx.get_maps(0, sig, "H"), ref["H"][sig])
        gptr, G, Q = ref["GQ"][sig]
        np.testing.assert_array_equal(ctx.get_maps(0, sig, "GQ_PTR"), gptr)
        np.testing.assert_array_equal(ctx.get_maps(0, sig, "Q"), Q)
        for tau in range(R):
            np.testing.assert_array_equal(ctx.get_maps(tau, sig, "I"), ref["I"][(sig, tau)])


def f32_ulp_distance(a, b):
    """|a - b| in units of fp32 ulp (ordered-integer distance)."""
    ai = np.asarray(a, np.float32).view(np.int32).astype(np.int64)
    bi = np.asarray(b, np.float32).view(np.int32).astype(np.int64)
    ai = np.where(ai < 0, -(ai & 0x7FFFFFFF), ai)
    bi = np.where(bi < 0, -(bi & 0x7FFFFFFF), bi)
    return np.abs(ai - bi)


def bf16_round(w32):
    """Round-to-nearest-even fp32 -> bf16, returned as fp32."""
    u = np.asarray(w32, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32)


def compare_rank(got, ref, fmt="f32", max_ulp=4):
    np.testing.assert_array_equal(got["row_ptr"], ref["row_ptr"])
    np.testing.assert_array_equal(got["tgt"].astype(np.int64), ref["tgt"])
    np.testing.assert_array_equal(got["d"].astype(np.int64), ref["d"])
    w32 = ref["w"].astype(np.float32)
    if fmt == "f32":
        u = f32_ulp_distance(got["w"], w32)
        assert u.max(initial=0) <= max_ulp, f"max ulp {u.max()}"
    elif fmt == "bf16":
        # bf16 of the GPU's fp32 draw vs bf16 of the oracle's: equal or one bf16 ulp apart
        ref16 = bf16_round(w32)
        d16 = np.abs(got["w"].view(np.int32).astype(np.int64) - ref16.view(np.int32).astype(np.int64)) >> 16
        assert d16.max(initial=0) <= 1
    else:
        rel = np.abs(got["w"] - w32) / np.maximum(np.abs(w32), 1e-30)
        assert rel.max(initial=0) <= 2.0 ** -10
    return True
