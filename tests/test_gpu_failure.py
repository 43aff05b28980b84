"""Failure detection without a GPU fault: bounded device waits report a timeout status,
host-side validation rejects bad input, and an allocator that fails returns ENOMEM."""
import ctypes as C

import pytest

from gpu_helpers import ensure_lib
from paper_2512_09502_gb300 import _lib, workloads as wl


@pytest.mark.gpu
def test_bounded_wait_gives_up_with_etimeout():
    lib = ensure_lib()
    assert lib.snn_selftest_bounded_wait(None) == -4          # SNN_ETIMEOUT
    # the device stays usable afterwards
    ctx = _lib.build_network(wl.tiny(wl.RULE_FIXED_INDEGREE, 5))
    ctx.calibrate()
    assert ctx.stats()["n_synapses"] == 100


@pytest.mark.gpu
def test_failing_allocator_returns_enomem():
    ensure_lib()
    calls = {"n": 0}

    class Failing(_lib.TorchAllocator):
        def __init__(self):
            super().__init__(0)
            inner = self._a

            def _alloc(user, nbytes, stream):
                calls["n"] += 1
                return 0 if calls["n"] > 5 else inner(user, nbytes, stream)
            self._a = _lib.snn_allocator._fields_[0][1](_alloc)
            self.struct = _lib.snn_allocator(self._a, self._f, None)

    ctx = _lib.build_network(wl.balanced(300, 75, 40, 10, wl.DELAY_NORMAL), allocator=Failing())
    with pytest.raises(_lib.SnnError) as e:
        ctx.calibrate()
    assert e.value.code == -2                                 # SNN_ENOMEM
    ctx.destroy()


@pytest.mark.gpu
@pytest.mark.parametrize("bad", ["delay_above_255", "clip_step_above_255", "range", "after_calibrate"])
def test_invalid_arguments_rejected(bad):
    ensure_lib()
    ctx = _lib.Context()
    ctx.create_population(100, wl.BALANCED_PARAMS)
    rule = wl.Rule(wl.RULE_FIXED_INDEGREE, 3)
    if bad == "delay_above_255":
        pr = wl.Projection(0, 100, 0, 100, rule, wl.Dist(wl.W_CONST, 1.0), wl.Dist(wl.D_NORMAL_MIN, 25.0, 2.0, 0.1), 1)
    elif bad == "clip_step_above_255":
        # clipped below at 30 ms (300 steps) with the normal's mass far below: every delay
        # would be the clip step, which a u8 delay cannot hold
        pr = wl.Projection(0, 100, 0, 100, rule, wl.Dist(wl.W_CONST, 1.0), wl.Dist(wl.D_NORMAL_MIN, 1.5, 0.75, 30.0), 1)
    elif bad == "range":
        pr = wl.Projection(0, 101, 0, 100, rule, wl.Dist(wl.W_CONST, 1.0), wl.Dist(wl.D_CONST, 1.0), 1)
    else:
        ctx.calibrate()
        pr = wl.Projection(0, 100, 0, 100, rule, wl.Dist(wl.W_CONST, 1.0), wl.Dist(wl.D_CONST, 1.0), 1)
    with pytest.raises(_lib.SnnError) as e:
        ctx.connect(pr)
    assert e.value.code == (-5 if bad == "after_calibrate" else -1)
