"""Thin ctypes binding of libsnn.so (include/snn.h): same names, argument marshalling
only.  Every step of construction and simulation runs in the library's CUDA kernels;
there is no Python or CPU fallback -- ``load()`` raises when the compiled library is
missing, and every call that returns a non-zero status raises ``SnnError``.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsnn.so")

SNN_OK = 0
SNN_EINVAL, SNN_ENOMEM, SNN_ECUDA, SNN_ETIMEOUT, SNN_ESTATE, SNN_EOVERFLOW = -1, -2, -3, -4, -5, -6
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ESTATE", -6: "EOVERFLOW"}
RULES = {"fixed_indegree": 0, "fixed_total": 1, "pairwise_bernoulli": 2, "pairwise_bernoulli_geometric": 3,
         "one_to_one": 4, "all_to_all": 5}
W_KINDS = {"const": 0, "normal_sign": 1}
D_KINDS = {"const": 0, "normal_min": 1}
WEIGHT_FORMATS = {"f32": 0, "bf16": 1, "f16": 2}
MAPS = {"R": 0, "L": 1, "S": 2, "T": 3, "P": 4, "TP_PTR": 5, "H": 6, "I": 7, "Q": 8, "GQ_PTR": 9}

EXPORTED = ["snn_create", "snn_destroy", "snn_last_error", "snn_create_population", "snn_connect",
            "snn_remote_connect", "snn_set_poisson_drive", "snn_calibrate", "snn_simulate",
            "snn_get_spikes", "snn_get_state", "snn_get_connections", "snn_get_row", "snn_get_maps",
            "snn_get_delay_table", "snn_stats", "snn_selftest_bounded_wait", "snn_connect_sorted_noalloc",
            "snn_ring_reduction_probe"]


class SnnError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} -> {STATUS.get(code, code)}: {msg}")
        self.code = code


class snn_allocator(C.Structure):
    _fields_ = [("alloc", C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)),
                ("user", C.c_void_p)]


class snn_config(C.Structure):
    _fields_ = [("dt_ms", C.c_double), ("n_ranks", C.c_uint32), ("weight_format", C.c_int32),
                ("exchange", C.c_int32), ("use_graph", C.c_int32),
                ("spike_log_capacity", C.c_uint64), ("radix_bits", C.c_int32), ("device", C.c_int32),
                ("profile_kernels", C.c_int32), ("sort_items", C.c_int32), ("deliver_ctas_per_sm", C.c_int32),
                ("dry_run", C.c_int32), ("dry_run_rank", C.c_uint32), ("xi", C.c_double),
                ("deliver_mode", C.c_int32)]


class snn_iaf_psc_exp_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ["tau_m", "C_m", "tau_syn_ex", "tau_syn_in", "V_th", "V_reset",
                                          "t_ref", "I_e", "V_init_lo", "V_init_hi"]] + \
               [("v_init_seed", C.c_uint64)]


class snn_rule(C.Structure):
    _fields_ = [("kind", C.c_int32), ("param", C.c_double)]


class snn_dist(C.Structure):
    _fields_ = [("kind", C.c_int32), ("mean", C.c_double), ("sd", C.c_double), ("lo", C.c_double)]


class snn_stats_t(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ["n_neurons", "n_synapses", "n_images", "n_blocks", "n_projections",
                                          "n_spikes", "n_events", "steps_done", "device_bytes",
                                          "peak_device_bytes", "spike_log_overflow"]] + \
               [(n, C.c_double) for n in ["t_generate_ms", "t_sort_ms", "t_finalize_ms", "t_maps_ms",
                                          "t_calibrate_ms", "t_simulate_ms"]] + \
               [(n, C.c_uint32) for n in ["sort_passes", "radix_bits", "key_bits", "ring_slots",
                                          "gen_kernel_launches", "sort_kernel_launches"]] + \
               [(n, C.c_uint64) for n in ["kernel_launches", "h2d_bytes", "d2h_bytes"]] + \
               [(n, C.c_double) for n in ["t_sort_pass_ms", "t_update_ms", "t_deliver_ms"]] + \
               [(n, C.c_uint64) for n in ["update_launches", "deliver_launches"]]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib: Optional[C.CDLL] = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libsnn.so (built by ``paper_2512_09502_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsnn.so not built ({path}); run __graft_entry__.build() -- "
                           "there is no CPU fallback")
    lib = C.CDLL(path)
    P = C.POINTER
    ctx = C.c_void_p
    sig = {
        "snn_create": ([P(snn_config), P(snn_allocator), C.c_void_p, P(ctx)], C.c_int),
        "snn_destroy": ([ctx], None),
        "snn_last_error": ([ctx], C.c_char_p),
        "snn_create_population": ([ctx, C.c_uint32, P(snn_iaf_psc_exp_params), P(C.c_uint32)], C.c_int),
        "snn_connect": ([ctx, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, P(snn_rule), P(snn_dist),
                         P(snn_dist), C.c_uint64, P(C.c_uint32)], C.c_int),
        "snn_remote_connect": ([ctx, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                C.c_uint32, C.c_uint32, P(snn_rule), P(snn_dist), P(snn_dist), C.c_int32,
                                C.c_uint64, P(C.c_uint32)], C.c_int),
        "snn_set_poisson_drive": ([ctx, C.c_uint32, C.c_uint32, C.c_double, C.c_double, C.c_uint64], C.c_int),
        "snn_calibrate": ([ctx], C.c_int),
        "snn_simulate": ([ctx, C.c_uint32], C.c_int),
        "snn_get_spikes": ([ctx, C.c_void_p, C.c_void_p, C.c_uint64, P(C.c_uint64)], C.c_int),
        "snn_get_state": ([ctx, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
        "snn_get_connections": ([ctx, C.c_uint32, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_uint64, P(C.c_uint64), P(C.c_uint64)], C.c_int),
        "snn_get_row": ([ctx, C.c_uint32, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64,
                         P(C.c_uint64)], C.c_int),
        "snn_get_maps": ([ctx, C.c_uint32, C.c_uint32, C.c_int32, C.c_void_p, C.c_uint64, P(C.c_uint64)], C.c_int),
        "snn_get_delay_table": ([ctx, C.c_uint32, C.c_void_p, C.c_uint64, P(C.c_uint64), P(C.c_uint32)], C.c_int),
        "snn_stats": ([ctx, P(snn_stats_t)], C.c_int),
        "snn_selftest_bounded_wait": ([C.c_void_p], C.c_int),
        "snn_ring_reduction_probe": ([ctx, C.c_int32, C.c_uint64, C.c_uint32, P(C.c_double)], C.c_int),
        "snn_connect_sorted_noalloc": ([C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, P(snn_rule),
                                        P(snn_dist), P(snn_dist), C.c_uint64, C.c_double, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_uint64, P(C.c_uint64), C.c_void_p,
                                        C.c_char_p, C.c_size_t], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class TorchAllocator:
    """snn_allocator backed by PyTorch's caching allocator (device memory plumbing)."""

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(user, nbytes, stream):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0))
            except Exception:      # out of memory -> NULL -> SNN_ENOMEM
                return 0

        def _free(user, ptr, nbytes, stream):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self._a = snn_allocator._fields_[0][1](_alloc)
        self._f = snn_allocator._fields_[1][1](_free)
        self.struct = snn_allocator(self._a, self._f, None)


class Context:
    """One snn_ctx.  Methods are named after the C entry points (minus the prefix)."""

    def __init__(self, *, dt: float = 0.1, n_ranks: int = 1, weight_format: str = "f32",
                 exchange: str = "p2p", use_graph: bool = True, spike_log_capacity: int = 0,
                 radix_bits: int = 0, device: int = 0, allocator: Optional[TorchAllocator] = None,
                 stream: Optional[int] = None, profile_kernels: int = 0, sort_items: int = 0,
                 deliver_ctas_per_sm: int = 0, dry_run_rank: Optional[int] = None, xi: float = 0.0,
                 deliver_mode: Optional[int] = None):
        self.lib = load()
        if not (radix_bits and sort_items and deliver_ctas_per_sm):
            from . import autotune        # tuned launch parameters, when a cache exists
            tuned = autotune.load() or {}
            radix_bits = radix_bits or int(tuned.get("radix_bits", 0))
            sort_items = sort_items or int(tuned.get("sort_items", 0))
            deliver_ctas_per_sm = deliver_ctas_per_sm or int(tuned.get("deliver_ctas_per_sm", 0))
            if deliver_mode is None:
                deliver_mode = int(tuned.get("deliver_mode", 0))
        if deliver_mode is None:
            deliver_mode = 0
        cfg = snn_config(dt, n_ranks, WEIGHT_FORMATS[weight_format], 0 if exchange == "p2p" else 1,
                         1 if use_graph else 0, spike_log_capacity, radix_bits, device,
                         int(profile_kernels), sort_items, deliver_ctas_per_sm,
                         0 if dry_run_rank is None else 1, 0 if dry_run_rank is None else dry_run_rank,
                         float(xi), int(deliver_mode))
        self._allocator = allocator
        h = C.c_void_p()
        rc = self.lib.snn_create(C.byref(cfg), C.byref(allocator.struct) if allocator else None,
                                 C.c_void_p(stream or 0), C.byref(h))
        if rc != SNN_OK:
            raise SnnError("snn_create", rc, "bad configuration or no CUDA device")
        self.h = h
        self.n_ranks = n_ranks
        self.weight_format = weight_format

    def _check(self, fn: str, rc: int):
        if rc != SNN_OK:
            raise SnnError(fn, rc, self.lib.snn_last_error(self.h).decode())

    def destroy(self):
        if self.h:
            self.lib.snn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    # ---- construction ----
    def create_population(self, n: int, params) -> int:
        p = snn_iaf_psc_exp_params(params.tau_m, params.C_m, params.tau_syn_ex, params.tau_syn_in,
                                   params.V_th, params.V_reset, params.t_ref, params.I_e,
                                   params.V_init_lo, params.V_init_hi, params.v_init_seed)
        first = C.c_uint32()
        self._check("snn_create_population", self.lib.snn_create_population(self.h, n, C.byref(p), C.byref(first)))
        return first.value

    @staticmethod
    def _dist(d, kinds):
        return snn_dist(kinds[d.kind], d.mean, d.sd, d.lo)

    def connect(self, pr) -> int:
        rule = snn_rule(RULES[pr.rule.kind], float(pr.rule.param))
        w, d = self._dist(pr.weight, W_KINDS), self._dist(pr.delay, D_KINDS)
        pid = C.c_uint32()
        if pr.src_stride == 1 and pr.tgt_stride == 1:
            rc = self.lib.snn_connect(self.h, pr.src_first, pr.n_src, pr.tgt_first, pr.n_tgt, C.byref(rule),
                                      C.byref(w), C.byref(d), pr.seed, C.byref(pid))
            self._check("snn_connect", rc)
        else:
            R = self.n_ranks
            assert pr.src_stride == R and pr.tgt_stride == R
            rc = self.lib.snn_remote_connect(self.h, pr.src_first % R, pr.src_first // R, pr.n_src,
                                             pr.tgt_first % R, pr.tgt_first // R, pr.n_tgt, 0,
                                             C.byref(rule), C.byref(w), C.byref(d), -1, pr.seed, C.byref(pid))
            self._check("snn_remote_connect", rc)
        return pid.value

    def set_poisson_drive(self, dr):
        self._check("snn_set_poisson_drive",
                    self.lib.snn_set_poisson_drive(self.h, dr.first, dr.n, dr.rate_hz, dr.weight, dr.seed))

    def calibrate(self):
        self._check("snn_calibrate", self.lib.snn_calibrate(self.h))

    def simulate(self, steps: int):
        self._check("snn_simulate", self.lib.snn_simulate(self.h, steps))

    # ---- results ----
    def get_spikes(self):
        n = C.c_uint64()
        self._check("snn_get_spikes", self.lib.snn_get_spikes(self.h, None, None, 0, C.byref(n)))
        st = np.zeros(n.value, np.uint32)
        gid = np.zeros(n.value, np.uint32)
        self._check("snn_get_spikes", self.lib.snn_get_spikes(self.h, _ptr(st), _ptr(gid), n.value, C.byref(n)))
        return st, gid

    def get_state(self, first: int, n: int):
        V, Ie, Ii = (np.zeros(n, np.float32) for _ in range(3))
        self._check("snn_get_state", self.lib.snn_get_state(self.h, first, n, _ptr(V), _ptr(Ie), _ptr(Ii)))
        return V, Ie, Ii

    def get_connections(self, rank: int = 0):
        nr, ns = C.c_uint64(), C.c_uint64()
        self._check("snn_get_connections", self.lib.snn_get_connections(
            self.h, rank, None, 0, None, None, None, 0, C.byref(nr), C.byref(ns)))
        rp = np.zeros(nr.value + 1, np.uint64)
        tgt = np.zeros(ns.value, np.uint32)
        w = np.zeros(ns.value, np.float32)
        d = np.zeros(ns.value, np.uint8)
        self._check("snn_get_connections", self.lib.snn_get_connections(
            self.h, rank, _ptr(rp), len(rp), _ptr(tgt), _ptr(w), _ptr(d), ns.value, C.byref(nr), C.byref(ns)))
        return dict(row_ptr=rp.astype(np.int64), tgt=tgt, w=w, d=d)

    def get_row(self, rank: int, row: int):
        n = C.c_uint64()
        self._check("snn_get_row", self.lib.snn_get_row(self.h, rank, row, None, None, None, 0, C.byref(n)))
        tgt = np.zeros(n.value, np.uint32)
        w = np.zeros(n.value, np.float32)
        d = np.zeros(n.value, np.uint8)
        self._check("snn_get_row", self.lib.snn_get_row(self.h, rank, row, _ptr(tgt), _ptr(w), _ptr(d),
                                                        n.value, C.byref(n)))
        return tgt, w, d

    def get_maps(self, tau: int, sigma: int, which: str):
        n = C.c_uint64()
        self._check("snn_get_maps", self.lib.snn_get_maps(self.h, tau, sigma, MAPS[which], None, 0, C.byref(n)))
        buf = np.zeros(n.value, np.int64)
        self._check("snn_get_maps", self.lib.snn_get_maps(self.h, tau, sigma, MAPS[which], _ptr(buf), n.value,
                                                          C.byref(n)))
        return buf

    def get_delay_table(self, proj_id: int):
        n, smin = C.c_uint64(), C.c_uint32()
        self._check("snn_get_delay_table", self.lib.snn_get_delay_table(self.h, proj_id, None, 0, C.byref(n),
                                                                        C.byref(smin)))
        buf = np.zeros(n.value, np.uint32)
        self._check("snn_get_delay_table", self.lib.snn_get_delay_table(self.h, proj_id, _ptr(buf), n.value,
                                                                        C.byref(n), C.byref(smin)))
        return smin.value, buf

    def ring_reduction_probe(self, mode: int, n_events: int, reps: int) -> float:
        """Mean ms per launch of the delivery's ceiling probe (snn_ring_reduction_probe)."""
        ms = C.c_double()
        self._check("snn_ring_reduction_probe",
                    self.lib.snn_ring_reduction_probe(self.h, mode, n_events, reps, C.byref(ms)))
        return ms.value

    def stats(self) -> dict:
        s = snn_stats_t()
        self._check("snn_stats", self.lib.snn_stats(self.h, C.byref(s)))
        return s.as_dict()


def build_network(net, **kw) -> Context:
    """Create a context and issue the create/connect/drive calls of a workload
    description (paper_2512_09502_gb300.workloads.Network).  Does not calibrate."""
    kw.setdefault("n_ranks", net.n_ranks)
    kw.setdefault("dt", net.dt)
    ctx = Context(**kw)
    for pop in net.populations:
        ctx.create_population(pop.n, pop.params)
    for pr in net.projections:
        ctx.connect(pr)
    for dr in net.drives:
        ctx.set_poisson_drive(dr)
    return ctx
