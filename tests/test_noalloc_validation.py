"""Argument checks of the allocation-free entry point, on the host (no GPU and no CUDA
call: every request below is rejected before the device is touched)."""
import ctypes as C

import pytest

from paper_2512_09502_gb300 import _lib, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _call(lib, n_neurons, n_tgt, rule_kind, param, delay):
    rule = _lib.snn_rule(_lib.RULES[rule_kind], float(param))
    wd = _lib.snn_dist(_lib.W_KINDS["const"], 1.0, 0.0, 0.0)
    dd = _lib.snn_dist(_lib.D_KINDS[delay[0]], *delay[1:])
    n = C.c_uint64()
    msg = C.create_string_buffer(256)
    # device pointers are never dereferenced on these paths
    fake = C.c_void_p(256)
    rc = lib.snn_connect_sorted_noalloc(n_neurons, 0, n_neurons, 0, n_tgt, C.byref(rule), C.byref(wd),
                                        C.byref(dd), 1, 0.1, fake, fake, fake, fake, 1 << 20, C.byref(n),
                                        None, msg, len(msg))
    return rc, msg.value.decode()


def test_huge_indegree_does_not_wrap(lib):
    """K = 2^62 + 1 on 4 targets: K * n_tgt wraps a 64-bit product to a small number, so
    the limit must be checked before the product."""
    rc, msg = _call(lib, 10, 4, "fixed_indegree", float(2 ** 62 + 1), ("const", 1.0, 0.0, 0.0))
    assert rc == _lib.SNN_EINVAL and "limit" in msg


@pytest.mark.parametrize("param", [1e30, float("inf"), float("nan"), 0.5, 0.0])
def test_out_of_range_parameters(lib, param):
    for kind in ("fixed_indegree", "fixed_total"):
        rc, _ = _call(lib, 10, 4, kind, param, ("const", 1.0, 0.0, 0.0))
        assert rc == _lib.SNN_EINVAL


def test_delay_clipped_above_255_steps_is_rejected(lib):
    """Normal(1.5, 0.75) ms clipped below at 30 ms with dt = 0.1 ms: every delay would be
    the 300-step clip value, which a u8 delay cannot hold."""
    rc, msg = _call(lib, 10, 4, "fixed_indegree", 2, ("normal_min", 1.5, 0.75, 30.0))
    assert rc == _lib.SNN_EINVAL and "255" in msg


def test_constant_delay_above_255_steps_is_rejected(lib):
    rc, msg = _call(lib, 10, 4, "fixed_indegree", 2, ("const", 1e12, 0.0, 0.0))
    assert rc == _lib.SNN_EINVAL and "255" in msg
