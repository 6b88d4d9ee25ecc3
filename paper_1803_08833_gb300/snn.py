"""Thin ctypes binding of libsnn.so (C ABI in include/snn.h).

Argument marshalling only: every step of the simulation runs in the library's
CUDA kernels.  PyTorch supplies the device memory (its caching allocator, via
the library's allocator hook) and the CUDA stream.  There is no fallback: if
libsnn.so is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# SNN_LIBRARY=check loads the checked build (device bounds checks, -DSNN_CHECK)
LIB_PATH = os.path.join(_PKG, "libsnn_check.so" if os.environ.get("SNN_LIBRARY") == "check" else "libsnn.so")

SNN_OK, SNN_EINVAL, SNN_ENOMEM, SNN_ECUDA, SNN_EOVERFLOW, SNN_ETIMEOUT, SNN_EBUDGET = 0, -1, -2, -3, -4, -5, -6
_STATUS = {0: "SNN_OK", -1: "SNN_EINVAL", -2: "SNN_ENOMEM", -3: "SNN_ECUDA", -4: "SNN_EOVERFLOW",
           -5: "SNN_ETIMEOUT", -6: "SNN_EBUDGET"}


class SnnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class SnnConfig(ctypes.Structure):
    _fields_ = [
        ("grid_w", ctypes.c_uint32), ("grid_h", ctypes.c_uint32),
        ("neurons_per_module", ctypes.c_uint32),
        ("exc_fraction", ctypes.c_float), ("spacing_um", ctypes.c_float),
        ("K", ctypes.c_uint32), ("kernel", ctypes.c_int32),
        ("sigma_um", ctypes.c_double), ("lambda_um", ctypes.c_double), ("cutoff_um", ctypes.c_double),
        ("w_exc_lo", ctypes.c_float), ("w_exc_hi", ctypes.c_float), ("w_inh", ctypes.c_float),
        ("d_exc_lo", ctypes.c_uint32), ("d_exc_hi", ctypes.c_uint32), ("d_inh", ctypes.c_uint32),
        ("tau_m_ms", ctypes.c_float), ("E_mV", ctypes.c_float), ("V_th_mV", ctypes.c_float),
        ("V_reset_mV", ctypes.c_float), ("t_ref_ms", ctypes.c_float),
        ("tau_c_ms", ctypes.c_float), ("alpha_c", ctypes.c_float), ("g_c_mV", ctypes.c_float),
        ("dt_ms", ctypes.c_float),
        ("ext_rate_hz", ctypes.c_float), ("J_ext_mV", ctypes.c_float),
        ("imposed_rate_hz", ctypes.c_float),
        ("weight_dtype", ctypes.c_int32), ("fx_shift", ctypes.c_uint32),
        ("seed", ctypes.c_uint64), ("raster_capacity", ctypes.c_uint64),
        ("table_layout", ctypes.c_int32),
        ("conn_rule", ctypes.c_int32), ("p_local", ctypes.c_float),
        ("A_remote", ctypes.c_double), ("p_min", ctypes.c_double),
        ("inh_local_only", ctypes.c_int32), ("weight_dist", ctypes.c_int32),
        ("w_exc_sd", ctypes.c_float), ("w_inh_sd", ctypes.c_float),
        ("delay_dist", ctypes.c_int32), ("delay_tau_ms", ctypes.c_float),
        ("stdp", ctypes.c_int32), ("stdp_A_plus", ctypes.c_float), ("stdp_A_minus", ctypes.c_float),
        ("stdp_tau_plus_ms", ctypes.c_float), ("stdp_tau_minus_ms", ctypes.c_float),
        ("stdp_w_max", ctypes.c_float), ("stdp_period_steps", ctypes.c_uint32),
    ]


class SnnStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("steps", "n_spikes", "rec_events", "ext_events", "raster_count", "raster_capacity",
                 "neuron_phase_ns", "deliver_phase_ns")]


class RequestResult(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("steps", ctypes.c_uint64), ("n_spikes", ctypes.c_uint64),
                ("rec_events", ctypes.c_uint64), ("ext_events", ctypes.c_uint64),
                ("raster_hash", ctypes.c_uint64), ("state_hash", ctypes.c_uint64),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("status", ctypes.c_int32), ("raster_overflow", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("ticks", "launches", "rec_events", "ext_events", "steps", "busy_ns", "used_bytes")] + \
               [("active", ctypes.c_uint32), ("queued", ctypes.c_uint32)]


class ShardInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("n_shards", "index", "row0", "row1", "n0", "n1", "h0", "h1", "peer_lo", "peer_hi", "D", "t")] + \
               [("table_synapses", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def load():
    """Load the in-tree libsnn.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsnn.so not found at %s: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, P = ctypes.c_void_p, ctypes.POINTER
    st = ctypes.c_int
    sig = {
        "snn_build_network": (st, [P(SnnConfig), ALLOC_FN, FREE_FN, vp, vp, P(vp)]),
        "snn_step": (st, [vp, ctypes.c_uint32, vp]),
        "snn_read_spikes": (st, [vp, vp, vp, ctypes.c_size_t, P(ctypes.c_size_t), vp]),
        "snn_clear_raster": (st, [vp, vp]),
        "snn_get_stats": (st, [vp, P(SnnStats), vp]),
        "snn_snapshot": (st, [vp, vp, ctypes.c_size_t, P(ctypes.c_size_t), vp]),
        "snn_restore": (st, [vp, vp, ctypes.c_size_t, vp]),
        "snn_get_table": (st, [vp, vp, vp, vp, vp]),
        "snn_get_rows": (st, [vp, ctypes.c_uint32, ctypes.c_uint32, vp, vp, vp, vp]),
        "snn_get_segments": (st, [vp, ctypes.c_uint32, ctypes.c_uint32, vp, P(ctypes.c_uint32), vp]),
        "snn_get_row_lengths": (st, [vp, ctypes.c_uint32, ctypes.c_uint32, vp, vp]),
        "snn_construction_tables": (st, [P(SnnConfig), vp, vp, P(ctypes.c_uint32), vp, vp, vp, ctypes.c_uint32,
                                         P(ctypes.c_uint32)]),
        "snn_get_cdf": (st, [vp, vp, vp, vp, P(ctypes.c_uint32), vp]),
        "snn_get_state": (st, [vp, vp, vp, vp, vp, P(ctypes.c_uint32), vp]),
        "snn_set_state": (st, [vp, vp, vp, vp, vp]),
        "snn_get_dims": (st, [vp, P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32),
                              P(ctypes.c_uint64)]),
        "snn_set_schedule": (st, [vp, ctypes.c_int32, ctypes.c_int32]),
        "snn_batch_set_shape": (st, [vp, ctypes.c_int32]),
        "snn_batch_set_layout": (st, [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64]),
        "snn_server_set_batch": (st, [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64]),
        "snn_batch_autotune": (st, [vp, ctypes.c_uint32, ctypes.c_char_p, P(ctypes.c_int32), P(ctypes.c_int32),
                                    P(ctypes.c_uint64), P(ctypes.c_double), P(ctypes.c_double), vp]),
        "snn_get_stdp": (st, [vp, vp, vp, vp, vp]),
        "snn_shard_build": (st, [P(SnnConfig), ctypes.c_uint32, ctypes.c_uint32, ALLOC_FN, FREE_FN, vp, vp, P(vp)]),
        "snn_shard_info": (st, [vp, P(ShardInfo)]),
        "snn_shard_integrate": (st, [vp, vp]),
        "snn_shard_outbox": (st, [vp, P(vp), P(vp)]),
        "snn_shard_deliver": (st, [vp, P(vp), P(vp), ctypes.c_uint32, vp]),
        "snn_shards_run": (st, [P(vp), ctypes.c_uint32, ctypes.c_uint32, vp]),
        "snn_shard_read_spikes": (st, [vp, vp, vp, ctypes.c_size_t, P(ctypes.c_size_t), vp]),
        "snn_shard_get_state": (st, [vp, vp, vp, vp, vp, vp]),
        "snn_shard_stats": (st, [vp, P(SnnStats), vp]),
        "snn_shard_destroy": (None, [vp]),
        "snn_set_bands": (st, [vp, ctypes.c_uint32, P(ctypes.c_uint32), vp]),
        "snn_set_window": (st, [vp, ctypes.c_uint32, ctypes.c_uint32, P(ctypes.c_uint32), P(ctypes.c_uint32), vp]),
        "snn_set_pull_window": (st, [vp, ctypes.c_uint32, ctypes.c_int32, P(ctypes.c_uint32), P(ctypes.c_int32), vp]),
        "snn_autotune": (st, [vp, ctypes.c_uint32, ctypes.c_char_p, P(ctypes.c_int32), P(ctypes.c_int32),
                              P(ctypes.c_double), vp]),
        "snn_set_timing": (st, [vp, ctypes.c_int32]),
        "snn_kernel_time": (st, [vp, ctypes.c_int32, P(ctypes.c_double), P(ctypes.c_uint64)]),
        "snn_set_wait_limit": (st, [vp, ctypes.c_uint64]),
        "snn_set_barrier_extra": (st, [vp, ctypes.c_uint32]),
        "snn_clear_error": (st, [vp, vp]),
        "snn_build_cdf_static": (st, [P(SnnConfig), vp, vp, vp, P(ctypes.c_uint32), vp]),
        "snn_launch_count": (ctypes.c_uint64, []),
        "snn_batch_create": (st, [P(vp), ctypes.c_uint32, ALLOC_FN, FREE_FN, vp, P(vp)]),
        "snn_batch_step": (st, [vp, P(ctypes.c_uint32), vp]),
        "snn_batch_set_graph": (st, [vp, ctypes.c_int32]),
        "snn_batch_waves": (st, [vp, P(ctypes.c_uint32), P(ctypes.c_uint64)]),
        "snn_batch_set_ring_budget": (st, [vp, ctypes.c_uint64]),
        "snn_set_resident_state": (st, [vp, ctypes.c_int32, P(ctypes.c_int32), vp]),
        "snn_batch_set_mode": (st, [vp, ctypes.c_int32]),
        "snn_batch_groups": (st, [vp, P(ctypes.c_uint32)]),
        "snn_plan_groups": (st, [vp, vp, ctypes.c_uint32, ctypes.c_uint32, vp]),
        "snn_plan_pull_bands": (st, [P(SnnConfig), ctypes.c_uint32, ctypes.c_int32, vp, vp, vp, ctypes.c_uint32,
                                     P(ctypes.c_uint32)]),
        "snn_batch_time": (st, [vp, P(ctypes.c_double), P(ctypes.c_uint64)]),
        "snn_batch_destroy": (None, [vp]),
        "snn_estimate_bytes": (ctypes.c_uint64, [P(SnnConfig)]),
        "snn_now_ns": (ctypes.c_uint64, []),
        "snn_server_create": (st, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ALLOC_FN, FREE_FN, vp, vp,
                                   P(vp)]),
        "snn_server_submit": (st, [vp, P(SnnConfig), ctypes.c_uint32, ctypes.c_uint64, P(ctypes.c_uint64)]),
        "snn_server_tick": (st, [vp, P(ctypes.c_uint32), P(ctypes.c_uint32)]),
        "snn_server_poll": (st, [vp, vp, ctypes.c_uint32, P(ctypes.c_uint32)]),
        "snn_server_stats": (st, [vp, vp]),
        "snn_server_destroy": (None, [vp]),
        "snn_destroy": (None, [vp]),
        "snn_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status):
    if status != SNN_OK:
        raise SnnError(status, load().snn_last_error().decode(errors="replace"))
    return status


def config(cfg: dict, raster_capacity: int = 0) -> SnnConfig:
    """Marshal a workload dictionary (keys = snn_config field names) into snn_config."""
    c = SnnConfig()
    names = {f[0] for f in SnnConfig._fields_}
    for k, v in cfg.items():
        if k == "kernel":
            v = {"gauss": 0, "exp": 1}.get(v, v)
        elif k == "weight_dtype":
            v = {"f32": 0, "bf16": 1}.get(v, v)
        elif k == "table_layout":
            v = {"draw": 0, "grouped": 1}.get(v, v)
        elif k == "conn_rule":
            v = {"fixed_k": 0, "pairwise": 1}.get(v, v)
        elif k == "weight_dist":
            v = {"uniform": 0, "gauss": 1}.get(v, v)
        elif k == "delay_dist":
            v = {"uniform": 0, "exp": 1}.get(v, v)
        if k not in names:
            raise KeyError("unknown snn_config field %r" % k)
        setattr(c, k, v)
    if raster_capacity:
        c.raster_capacity = raster_capacity
    return c


def construction_tables(cfg: dict) -> dict:
    """The host-derived construction tables of a description (no GPU work):
    Gaussian efficacy quantiles, exponential delay thresholds, pairwise stencil."""
    L = load()
    c = config(cfg)
    nd, npair = ctypes.c_uint32(), ctypes.c_uint32()
    check(L.snn_construction_tables(ctypes.byref(c), None, None, ctypes.byref(nd), None, None, None, 0,
                                    ctypes.byref(npair)))
    wtab = np.zeros(2 * 4096, np.float32)
    dthr = np.zeros(max(1, nd.value), np.uint64)
    k = npair.value
    dx, dy, thr = np.zeros(max(1, k), np.int32), np.zeros(max(1, k), np.int32), np.zeros(max(1, k), np.uint64)
    check(L.snn_construction_tables(ctypes.byref(c), _ptr(wtab), _ptr(dthr), ctypes.byref(nd), _ptr(dx), _ptr(dy),
                                    _ptr(thr), max(1, k), ctypes.byref(npair)))
    return {"wtab_exc": wtab[:4096], "wtab_inh": wtab[4096:], "dthr": dthr[:nd.value],
            "pair_dx": dx[:k], "pair_dy": dy[:k], "pair_thr": thr[:k]}


def launch_count() -> int:
    return int(load().snn_launch_count())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class _TorchAllocator:
    """Allocator hook backed by PyTorch's caching allocator on one device/stream."""

    def __init__(self, device, stream):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, size, ctx):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(size), self.device, self.stream)
        except Exception:  # out of memory: the library reports SNN_ENOMEM
            return None

    def _free(self, ptr, ctx):
        self.torch.cuda.caching_allocator_delete(ptr)


class Network:
    """One simulated network resident on the current CUDA device."""

    def __init__(self, cfg: dict, raster_capacity: int = 1 << 20, stream=None, allocator="torch"):
        import torch
        L = load()
        self.cfg = dict(cfg)
        self._torch = torch
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._s = ctypes.c_void_p(self.stream.cuda_stream)
        self._c = config(cfg, raster_capacity)
        self._alloc = _TorchAllocator(self.device, self.stream) if allocator == "torch" else None
        h = ctypes.c_void_p()
        if self._alloc is not None:
            st = L.snn_build_network(ctypes.byref(self._c), self._alloc.alloc, self._alloc.free, None,
                                     self._s, ctypes.byref(h))
        else:
            st = L.snn_build_network(ctypes.byref(self._c), ALLOC_FN(), FREE_FN(), None, self._s,
                                     ctypes.byref(h))
        check(st)
        self._h = h
        N, K, D = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        nbytes = ctypes.c_uint64()
        check(L.snn_get_dims(h, ctypes.byref(N), ctypes.byref(K), ctypes.byref(D), ctypes.byref(nbytes)))
        self.N, self.K, self.D, self.device_bytes = N.value, K.value, D.value, nbytes.value
        self.raster_capacity = raster_capacity
        self.n_modules = int(cfg["grid_w"]) * int(cfg["grid_h"])

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load().snn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- simulation ------------------------------------------------------
    def step(self, n: int = 1):
        check(load().snn_step(self._h, int(n), self._s))

    def read_spikes(self, cap=None, allow_overflow=False):
        cap = self.raster_capacity if cap is None else cap
        steps = np.empty(cap, np.uint32)
        ids = np.empty(cap, np.uint32)
        n = ctypes.c_size_t()
        st = load().snn_read_spikes(self._h, _ptr(steps), _ptr(ids), cap, ctypes.byref(n), self._s)
        if not (allow_overflow and st == SNN_EOVERFLOW):
            check(st)
        return steps[: n.value], ids[: n.value]

    def read_spikes_into(self, steps: np.ndarray, ids: np.ndarray) -> int:
        """Copy the raster into caller-owned (e.g. pinned) host arrays; returns the count."""
        n = ctypes.c_size_t()
        check(load().snn_read_spikes(self._h, _ptr(steps), _ptr(ids), min(len(steps), len(ids)),
                                     ctypes.byref(n), self._s))
        return n.value

    def clear_raster(self):
        check(load().snn_clear_raster(self._h, self._s))

    def stats(self) -> dict:
        s = SnnStats()
        check(load().snn_get_stats(self._h, ctypes.byref(s), self._s))
        return {f[0]: int(getattr(s, f[0])) for f in SnnStats._fields_}

    # -- inspection --------------------------------------------------------
    def row_lengths(self, first: int = 0, count=None):
        """Out-degree of rows [first, first + count)."""
        count = self.N - first if count is None else count
        out = np.empty(max(1, count), np.uint32)
        check(load().snn_get_row_lengths(self._h, first, count, _ptr(out), self._s))
        return out[:count]

    def csr(self, first: int = 0, count=None):
        """Synapse rows [first, first + count) back to back as flat (target,
        weight, delay) arrays (row lengths: row_lengths())."""
        count = self.N - first if count is None else count
        ns = int(self.row_lengths(first, count).sum()) if count else 0
        tgt = np.empty(ns, np.uint32)
        w = np.empty(ns, np.float32)
        d = np.empty(ns, np.uint8)
        check(load().snn_get_rows(self._h, first, count, _ptr(tgt), _ptr(w), _ptr(d), self._s))
        return tgt, w, d

    def segments(self, first: int = 0, count=None):
        """Grouped layout: segment starts, shape (count, stride)."""
        count = self.N - first if count is None else count
        stride = ctypes.c_uint32()
        check(load().snn_get_segments(self._h, 0, 0, None, ctypes.byref(stride), self._s))
        out = np.empty(count * stride.value, np.uint16)
        check(load().snn_get_segments(self._h, first, count, _ptr(out), ctypes.byref(stride), self._s))
        return out.reshape(count, stride.value)

    def cdf(self):
        mo = ctypes.c_uint32()
        check(load().snn_get_cdf(self._h, None, None, None, ctypes.byref(mo), self._s))
        m = mo.value
        T = np.empty(self.n_modules * m, np.uint32)
        TM = np.empty(self.n_modules * m, np.uint32)
        cnt = np.empty(self.n_modules, np.uint32)
        check(load().snn_get_cdf(self._h, _ptr(T), _ptr(TM), _ptr(cnt), ctypes.byref(mo), self._s))
        return T.reshape(self.n_modules, m), TM.reshape(self.n_modules, m), cnt

    def state(self):
        V = np.empty(self.N, np.float32)
        c = np.empty(self.N, np.float32)
        ref = np.empty(self.N, np.uint8)
        ring = np.empty(self.D * self.N, np.int32)
        t = ctypes.c_uint32()
        check(load().snn_get_state(self._h, _ptr(V), _ptr(c), _ptr(ref), _ptr(ring), ctypes.byref(t), self._s))
        return {"V": V, "c": c, "ref": ref, "ring": ring.reshape(self.D, self.N), "t": t.value}

    def set_state(self, V=None, c=None, ref=None):
        V = None if V is None else np.ascontiguousarray(V, np.float32)
        c = None if c is None else np.ascontiguousarray(c, np.float32)
        ref = None if ref is None else np.ascontiguousarray(ref, np.uint8)
        check(load().snn_set_state(self._h, _ptr(V), _ptr(c), _ptr(ref), self._s))

    def snapshot(self) -> bytes:
        n = ctypes.c_size_t()
        check(load().snn_snapshot(self._h, None, 0, ctypes.byref(n), self._s))
        buf = ctypes.create_string_buffer(n.value)
        check(load().snn_snapshot(self._h, buf, n.value, ctypes.byref(n), self._s))
        return buf.raw

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        check(load().snn_restore(self._h, buf, len(blob), self._s))

    # -- tuning / timing ---------------------------------------------------
    def set_schedule(self, schedule: int, block: int = 0):
        """0/1: two launches per step; 2: persistent push kernel; 3: target
        tiles; 4: owned windows with record queues; 5: owned windows filled by
        pulling row ranges (rows grouped by target module: the grouped layout,
        or the per-pair law).  Results are identical."""
        check(load().snn_set_schedule(self._h, int(schedule), int(block)))

    def stdp(self):
        """(accumulated change of every synapse in 2^-16 mV units, rows back to
        back; post trace y; pre trace x) of a network with plasticity."""
        ln = self.row_lengths()
        delta = np.empty(int(ln.astype(np.int64).sum()), np.int32)
        y = np.empty(self.N, np.float32)
        x = np.empty(self.N, np.float32)
        check(load().snn_get_stdp(self._h, _ptr(delta), _ptr(y), _ptr(x), self._s))
        return delta, y, x

    def set_window(self, window: int = 0, queue_cap: int = 0):
        """Schedule 4's delay window (steps kept in shared memory per band) and
        record-queue capacity; 0 picks the default.  Returns (window, cap)."""
        w, c = ctypes.c_uint32(), ctypes.c_uint32()
        check(load().snn_set_window(self._h, int(window), int(queue_cap), ctypes.byref(w), ctypes.byref(c), self._s))
        return w.value, c.value

    def set_pull_window(self, window: int = 0, band_mode: int = 0) -> int:
        """Schedule 5's delay window (steps kept in shared memory per band; 0
        picks the most that fit) and bands (0 automatic, 1 uniform, 2 on module
        boundaries).  Returns the window in use (the band mode in use is
        `pull_band_mode`)."""
        w, m = ctypes.c_uint32(), ctypes.c_int32()
        check(load().snn_set_pull_window(self._h, int(window), int(band_mode), ctypes.byref(w), ctypes.byref(m),
                                         self._s))
        self.pull_band_mode = m.value
        return w.value

    def set_bands(self, bands: int = 0) -> int:
        """Banded delivery of schedule 2 (0 = automatic); returns the band count in use."""
        out = ctypes.c_uint32()
        check(load().snn_set_bands(self._h, int(bands), ctypes.byref(out), self._s))
        return out.value

    def set_resident_state(self, enable: bool = True) -> bool:
        """Neuron state in shared memory through each persistent launch (when it
        fits); returns whether the launches keep it resident."""
        out = ctypes.c_int32()
        check(load().snn_set_resident_state(self._h, 1 if enable else 0, ctypes.byref(out), self._s))
        return bool(out.value)

    def autotune(self, trial_steps: int = 20, cache_path=None):
        """Pick the fastest schedule (state unchanged); returns (schedule, block, ms per step)."""
        sc, bl, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        check(load().snn_autotune(self._h, int(trial_steps), None if cache_path is None else cache_path.encode(),
                                  ctypes.byref(sc), ctypes.byref(bl), ctypes.byref(ms), self._s))
        return sc.value, bl.value, ms.value

    def set_timing(self, every: int):
        """Bracket the kernels of every n-th step with CUDA events (0 = off)."""
        check(load().snn_set_timing(self._h, int(every)))

    def kernel_time(self) -> dict:
        """Summed CUDA-event time (ms) and timed launches per kernel."""
        out = {}
        for name, which in (("neuron", 0), ("deliver", 1), ("persistent", 2)):
            ms, n = ctypes.c_double(), ctypes.c_uint64()
            check(load().snn_kernel_time(self._h, which, ctypes.byref(ms), ctypes.byref(n)))
            out[name + "_ms"] = ms.value
            out[name + "_launches"] = n.value
        return out

    def set_wait_limit(self, ns: int):
        check(load().snn_set_wait_limit(self._h, int(ns)))

    def set_barrier_extra(self, extra: int):
        check(load().snn_set_barrier_extra(self._h, int(extra)))

    def clear_error(self):
        check(load().snn_clear_error(self._h, self._s))


class Batch:
    """Independent networks advanced together in one persistent launch."""

    def __init__(self, nets, stream=None):
        import torch
        L = load()
        self.nets = list(nets)
        n = len(self.nets)
        dev = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._s = ctypes.c_void_p(self.stream.cuda_stream)
        self._alloc = _TorchAllocator(dev, self.stream)
        arr = (ctypes.c_void_p * n)(*[net._h.value for net in self.nets])
        h = ctypes.c_void_p()
        check(L.snn_batch_create(arr, n, self._alloc.alloc, self._alloc.free, None, ctypes.byref(h)))
        self._h = h

    def step(self, steps):
        """steps: one count per network (0 = idle)."""
        n = len(self.nets)
        if isinstance(steps, int):
            steps = [steps] * n
        arr = (ctypes.c_uint32 * n)(*[int(x) for x in steps])
        check(load().snn_batch_step(self._h, arr, self._s))

    def set_graph(self, enable: bool):
        check(load().snn_batch_set_graph(self._h, 1 if enable else 0))

    def set_ring_budget(self, nbytes: int):
        check(load().snn_batch_set_ring_budget(self._h, int(nbytes)))

    def set_shape(self, shape: int):
        check(load().snn_batch_set_shape(self._h, int(shape)))

    def autotune(self, trial_steps: int = 100, cache_path=None):
        """Times every (layout, launch shape, ring budget) candidate and keeps
        the fastest; returns {mode, shape, ring_budget, ms_per_step}."""
        m, sh, bud, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_uint64(), ctypes.c_double()
        trials = (ctypes.c_double * 12)()
        cp = cache_path.encode() if cache_path else None
        check(load().snn_batch_autotune(self._h, int(trial_steps), cp, ctypes.byref(m), ctypes.byref(sh),
                                        ctypes.byref(bud), ctypes.byref(ms), trials, self._s))
        sweep = {}
        for k, t in enumerate(trials):
            if t >= 0:
                sweep["%s/shape%d/%.2fL2" % (("groups", "global")[k // 6], (k // 3) % 2, (0.35, 0.5, 0.65)[k % 3])] = t
        return {"mode": "global" if m.value == 1 else "groups", "shape": sh.value, "ring_budget": bud.value,
                "ms_per_step": ms.value, "sweep_ms_per_step": sweep}

    def set_mode(self, mode: str):
        """'groups' (default: every network of a wave on CTAs of its own) or
        'global' (one neuron and task space for the whole wave)."""
        check(load().snn_batch_set_mode(self._h, {"groups": 0, "global": 1}[mode]))

    def groups(self):
        """CTAs of each network's group in the last step call (0: idle, alone
        in its wave, or in a global wave)."""
        n = len(self.nets)
        arr = (ctypes.c_uint32 * n)()
        check(load().snn_batch_groups(self._h, arr))
        return list(arr)

    def waves(self):
        """(number of launches per step call, ring budget in bytes)."""
        w, r = ctypes.c_uint32(), ctypes.c_uint64()
        check(load().snn_batch_waves(self._h, ctypes.byref(w), ctypes.byref(r)))
        return w.value, r.value

    def time(self):
        ms, n = ctypes.c_double(), ctypes.c_uint64()
        check(load().snn_batch_time(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def close(self):
        if getattr(self, "_h", None):
            load().snn_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class _DeviceArray:
    """A 1-D int32 device buffer owned by the library, seen through the CUDA
    array interface (no copy)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<i4", "data": (int(ptr), False),
                                         "version": 3}


class Shard:
    """Shard `index` of an n-way decomposition of a network into stripes of
    module rows (the paper's spatial decomposition), on the current device."""

    def __init__(self, cfg: dict, n_shards: int, index: int, raster_capacity: int = 1 << 20, stream=None):
        import torch
        L = load()
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._s = ctypes.c_void_p(self.stream.cuda_stream)
        self._c = config(cfg, raster_capacity)
        self._alloc = _TorchAllocator(self.device, self.stream)
        h = ctypes.c_void_p()
        check(L.snn_shard_build(ctypes.byref(self._c), int(n_shards), int(index), self._alloc.alloc,
                                self._alloc.free, None, self._s, ctypes.byref(h)))
        self._h = h
        self.raster_capacity = raster_capacity

    def info(self) -> dict:
        i = ShardInfo()
        check(load().snn_shard_info(self._h, ctypes.byref(i)))
        return {f[0]: getattr(i, f[0]) for f in ShardInfo._fields_}

    def integrate(self):
        check(load().snn_shard_integrate(self._h, self._s))

    def outbox(self):
        """Device pointers (ids, count) of the step's spikes."""
        a, b = ctypes.c_void_p(), ctypes.c_void_p()
        check(load().snn_shard_outbox(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def outbox_tensors(self):
        """Zero-copy int32 tensor views of the outbox: (ids, capacity n1 - n0;
        count, 1 entry), for the exchange with other ranks."""
        import torch
        ids_p, cnt_p = self.outbox()
        inf = self.info()
        return (torch.as_tensor(_DeviceArray(ids_p, max(inf["n1"] - inf["n0"], 1)), device="cuda"),
                torch.as_tensor(_DeviceArray(cnt_p, 1), device="cuda"))

    def deliver(self, lists):
        """lists: (ids device pointer, count device pointer) per inbound list."""
        n = len(lists)
        ids = (ctypes.c_void_p * max(n, 1))(*[x[0] for x in lists])
        cnt = (ctypes.c_void_p * max(n, 1))(*[x[1] for x in lists])
        check(load().snn_shard_deliver(self._h, ids, cnt, n, self._s))

    def read_spikes(self):
        steps = np.empty(self.raster_capacity, np.uint32)
        ids = np.empty(self.raster_capacity, np.uint32)
        n = ctypes.c_size_t()
        check(load().snn_shard_read_spikes(self._h, _ptr(steps), _ptr(ids), self.raster_capacity, ctypes.byref(n),
                                           self._s))
        return steps[: n.value], ids[: n.value]

    def state(self):
        inf = self.info()
        Nl = inf["n1"] - inf["n0"]
        V, c = np.empty(Nl, np.float32), np.empty(Nl, np.float32)
        ref = np.empty(Nl, np.uint8)
        ring = np.empty(inf["D"] * Nl, np.int32)
        check(load().snn_shard_get_state(self._h, _ptr(V), _ptr(c), _ptr(ref), _ptr(ring), self._s))
        return {"V": V, "c": c, "ref": ref, "ring": ring.reshape(inf["D"], Nl)}

    def stats(self) -> dict:
        st = SnnStats()
        check(load().snn_shard_stats(self._h, ctypes.byref(st), self._s))
        return {f[0]: getattr(st, f[0]) for f in SnnStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().snn_shard_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ShardedNetwork:
    """All shards of an n-way decomposition on the current device, stepped by
    snn_shards_run (the exchange reads the peers' outboxes in place); the
    union state and raster are those of the undivided network."""

    def __init__(self, cfg: dict, n_shards: int, raster_capacity: int = 1 << 20, stream=None):
        self.cfg = dict(cfg)
        self.shards = [Shard(cfg, n_shards, k, raster_capacity, stream) for k in range(n_shards)]
        self._s = self.shards[0]._s
        self._arr = (ctypes.c_void_p * n_shards)(*[sh._h.value for sh in self.shards])

    def step(self, n: int = 1):
        check(load().snn_shards_run(self._arr, len(self.shards), int(n), self._s))

    def read_spikes(self):
        parts = [sh.read_spikes() for sh in self.shards]
        st = np.concatenate([p[0] for p in parts])
        ids = np.concatenate([p[1] for p in parts])
        order = np.lexsort((ids, st))
        return st[order], ids[order]

    def state(self):
        parts = [sh.state() for sh in self.shards]
        return {"V": np.concatenate([p["V"] for p in parts]), "c": np.concatenate([p["c"] for p in parts]),
                "ref": np.concatenate([p["ref"] for p in parts]),
                "ring": np.concatenate([p["ring"] for p in parts], axis=1)}

    def stats(self) -> dict:
        tot = {}
        for sh in self.shards:
            for k, v in sh.stats().items():
                tot[k] = tot.get(k, 0) + v
        tot["steps"] = self.shards[0].info()["t"]
        return tot

    def close(self):
        for sh in self.shards:
            sh.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def now_ns() -> int:
    """The library's host monotonic clock (time base of request arrivals)."""
    return int(load().snn_now_ns())


def plan_pull_bands(cfg: dict, sms: int, band_mode: int):
    """Schedule 5's bands and run tables for a description (host only):
    (bq, run_ptr, runs) with runs an (n, 2) array of {source module,
    j0 | j1 << 16}; band b owns the quads [bq[b], bq[b + 1])."""
    L = load()
    c = config(cfg)
    bq = np.zeros(sms + 1, np.uint32)
    ptr = np.zeros(sms + 1, np.uint32)
    n = ctypes.c_uint32()
    st_ = L.snn_plan_pull_bands(ctypes.byref(c), int(sms), int(band_mode), _ptr(bq), _ptr(ptr), None, 0,
                                ctypes.byref(n))
    if st_ not in (SNN_OK, SNN_EOVERFLOW):
        check(st_)
    runs = np.zeros((max(1, n.value), 2), np.uint32)
    check(L.snn_plan_pull_bands(ctypes.byref(c), int(sms), int(band_mode), _ptr(bq), _ptr(ptr), _ptr(runs),
                                max(1, n.value), ctypes.byref(n)))
    return bq, ptr, runs[:n.value]


def plan_groups(steps, work, ctas: int):
    """CTAs per network of a grouped batch wave (snn_plan_groups): steps and
    estimated work in CTA-microseconds per step, one per network."""
    s = np.ascontiguousarray(steps, dtype=np.uint32)
    w = np.ascontiguousarray(work, dtype=np.float64)
    if s.shape != w.shape:
        raise ValueError("steps and work differ in length")
    out = np.zeros(len(s), np.uint32)
    check(load().snn_plan_groups(_ptr(s), _ptr(w), len(s), int(ctas), _ptr(out)))
    return out


def estimate_bytes(cfg: dict, raster_capacity: int = 0) -> int:
    c = config(cfg, raster_capacity)
    return int(load().snn_estimate_bytes(ctypes.byref(c)))


class Server:
    """Continuous-batching simulation server (snn_server_* of the C ABI)."""

    def __init__(self, budget_bytes: int, chunk_steps: int = 250, max_slots: int = 128, stream=None):
        import torch
        dev = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._s = ctypes.c_void_p(self.stream.cuda_stream)
        self._alloc = _TorchAllocator(dev, self.stream)
        h = ctypes.c_void_p()
        check(load().snn_server_create(int(budget_bytes), int(chunk_steps), int(max_slots), self._alloc.alloc,
                                       self._alloc.free, None, self._s, ctypes.byref(h)))
        self._h = h

    def set_batch(self, mode: str = "groups", shape: int = 0, ring_budget: int = 0):
        """Layout of every tick's batch (e.g. a batch tuner's choice)."""
        check(load().snn_server_set_batch(self._h, 1 if mode == "global" else 0, int(shape), int(ring_budget)))

    def submit(self, cfg: dict, steps: int, arrival_ns: int = 0, raster_capacity: int = 1 << 16) -> int:
        c = config(cfg, raster_capacity)
        rid = ctypes.c_uint64()
        check(load().snn_server_submit(self._h, ctypes.byref(c), int(steps), int(arrival_ns), ctypes.byref(rid)))
        return rid.value

    def tick(self):
        a, q = ctypes.c_uint32(), ctypes.c_uint32()
        check(load().snn_server_tick(self._h, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def poll(self):
        out = []
        buf = (RequestResult * 256)()
        while True:
            n = ctypes.c_uint32()
            check(load().snn_server_poll(self._h, buf, 256, ctypes.byref(n)))
            out += [{f[0]: getattr(buf[i], f[0]) for f in RequestResult._fields_}
                    for i in range(n.value)]
            if n.value < 256:
                return out

    def stats(self) -> dict:
        st = ServerStats()
        check(load().snn_server_stats(self._h, ctypes.byref(st)))
        return {f[0]: getattr(st, f[0]) for f in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().snn_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
