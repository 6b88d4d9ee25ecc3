"""Correctness oracle for the DPSNN per-timestep method (Pastorelli et al., PDP 2018).

TEST INFRASTRUCTURE ONLY.  A plain, single-threaded C restatement of the method
(``snn_oracle.c``), loaded through ctypes.  Only ``tests/``, the smoke check and
the CPU-baseline leg of ``bench.py`` may import this package; the CUDA library
never does, and this package imports nothing from it.

Parity status: see the header of ``snn_oracle.h``.  Whole-network firing rates
are "parity unpinned" against the paper (its drive parameters are not given).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snn_oracle.c")
_HDR = os.path.join(_HERE, "snn_oracle.h")
_SO = os.path.join(_HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) if it is missing or stale."""
    stale = (not os.path.exists(_SO)) or any(
        os.path.getmtime(s) > os.path.getmtime(_SO) for s in (_SRC, _HDR))
    if force or stale:
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


class OrParams(ctypes.Structure):
    _fields_ = [
        ("grid_w", ctypes.c_uint32), ("grid_h", ctypes.c_uint32),
        ("neurons_per_module", ctypes.c_uint32),
        ("exc_fraction", ctypes.c_float), ("spacing_um", ctypes.c_float),
        ("K", ctypes.c_uint32), ("kernel", ctypes.c_int32),
        ("sigma_um", ctypes.c_double), ("lambda_um", ctypes.c_double),
        ("cutoff_um", ctypes.c_double),
        ("w_exc_lo", ctypes.c_float), ("w_exc_hi", ctypes.c_float), ("w_inh", ctypes.c_float),
        ("d_exc_lo", ctypes.c_uint32), ("d_exc_hi", ctypes.c_uint32), ("d_inh", ctypes.c_uint32),
        ("tau_m", ctypes.c_float), ("E", ctypes.c_float), ("V_th", ctypes.c_float),
        ("V_reset", ctypes.c_float), ("t_ref", ctypes.c_float), ("tau_c", ctypes.c_float),
        ("alpha_c", ctypes.c_float), ("g_c", ctypes.c_float), ("dt", ctypes.c_float),
        ("ext_rate_hz", ctypes.c_float), ("J_ext", ctypes.c_float),
        ("imposed_rate_hz", ctypes.c_float),
        ("weight_bf16", ctypes.c_int32), ("fx_shift", ctypes.c_uint32),
        ("seed", ctypes.c_uint64),
        ("conn_rule", ctypes.c_int32), ("p_local", ctypes.c_float),
        ("A_remote", ctypes.c_double), ("p_min", ctypes.c_double),
        ("inh_local_only", ctypes.c_int32), ("weight_dist", ctypes.c_int32),
        ("w_exc_sd", ctypes.c_float), ("w_inh_sd", ctypes.c_float),
        ("delay_dist", ctypes.c_int32), ("delay_tau_ms", ctypes.c_float),
        ("stdp", ctypes.c_int32), ("stdp_A_plus", ctypes.c_float), ("stdp_A_minus", ctypes.c_float),
        ("stdp_tau_plus_ms", ctypes.c_float), ("stdp_tau_minus_ms", ctypes.c_float),
        ("stdp_w_max", ctypes.c_float), ("stdp_period_steps", ctypes.c_uint32),
    ]


class OrConsts(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_uint32), ("n_modules", ctypes.c_uint32), ("n_exc", ctypes.c_uint32),
        ("D", ctypes.c_uint32), ("ref_steps", ctypes.c_uint32), ("R2", ctypes.c_uint32),
        ("max_offsets", ctypes.c_uint32),
        ("a_m", ctypes.c_float), ("a_c", ctypes.c_float), ("kc", ctypes.c_float),
        ("J_ext_fx", ctypes.c_int32), ("imposed_thresh", ctypes.c_uint64),
        ("pois_len", ctypes.c_uint32), ("pois", ctypes.c_uint64 * 64),
        ("n_pair_offsets", ctypes.c_uint32),
    ]


class OrConsts64(ctypes.Structure):
    _fields_ = [("a_m", ctypes.c_double), ("a_c", ctypes.c_double), ("kc", ctypes.c_double)]


# names used by workload dictionaries -> oracle field names
_MAP = {
    "tau_m_ms": "tau_m", "E_mV": "E", "V_th_mV": "V_th", "V_reset_mV": "V_reset",
    "t_ref_ms": "t_ref", "tau_c_ms": "tau_c", "g_c_mV": "g_c", "dt_ms": "dt",
    "J_ext_mV": "J_ext",
}
_IGNORED = {"raster_capacity", "weight_dtype", "table_layout"}


def params(cfg: dict) -> OrParams:
    p = OrParams()
    names = {f[0] for f in OrParams._fields_}
    for k, v in cfg.items():
        if k == "weight_dtype":
            p.weight_bf16 = 1 if v in ("bf16", 1) else 0
            continue
        if k == "kernel":
            p.kernel = {"gauss": 0, "exp": 1}.get(v, v)
            continue
        if k == "conn_rule":
            p.conn_rule = {"fixed_k": 0, "pairwise": 1}.get(v, v)
            continue
        if k == "weight_dist":
            p.weight_dist = {"uniform": 0, "gauss": 1}.get(v, v)
            continue
        if k == "delay_dist":
            p.delay_dist = {"uniform": 0, "exp": 1}.get(v, v)
            continue
        if k in _IGNORED:
            continue
        name = _MAP.get(k, k)
        if name not in names:
            raise KeyError("unknown parameter %r" % k)
        setattr(p, name, v)
    return p


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        u32p, u64p = P(ctypes.c_uint32), P(ctypes.c_uint64)
        L.or_philox.argtypes = [u32p, u32p, u32p]
        L.or_bf16_bits.argtypes = [ctypes.c_float]
        L.or_bf16_bits.restype = ctypes.c_uint16
        L.or_constants.argtypes = [P(OrParams), P(OrConsts)]
        L.or_cdf_table.argtypes = [P(OrParams), ctypes.c_uint32, u32p, u32p,
                                   P(ctypes.c_double), ctypes.c_uint32, u32p]
        L.or_lif_update.argtypes = [P(OrConsts), P(OrParams), P(ctypes.c_float),
                                    P(ctypes.c_float), P(ctypes.c_uint8), ctypes.c_int,
                                    ctypes.c_int32, ctypes.c_int]
        L.or_poisson_count.argtypes = [P(OrConsts), ctypes.c_uint32]
        L.or_poisson_count.restype = ctypes.c_uint32
        L.or_create.argtypes = [P(OrParams), ctypes.c_int]
        L.or_create.restype = ctypes.c_void_p
        L.or_destroy.argtypes = [ctypes.c_void_p]
        L.or_error.restype = ctypes.c_char_p
        L.or_n_synapses.argtypes = [ctypes.c_void_p]
        L.or_n_synapses.restype = ctypes.c_uint64
        L.or_get_csr.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.or_get_csr_f64.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.or_set_delivery_shuffle.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
        L.or_step.argtypes = [ctypes.c_void_p, ctypes.c_uint32]
        L.or_raster_size.argtypes = [ctypes.c_void_p]
        L.or_raster_size.restype = ctypes.c_uint64
        L.or_get_raster.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.or_clear_raster.argtypes = [ctypes.c_void_p]
        L.or_time.argtypes = [ctypes.c_void_p]
        L.or_time.restype = ctypes.c_uint32
        L.or_get_state.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 4
        L.or_get_state_f64.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 2
        L.or_get_stdp.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 3
        L.or_set_state_f64.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 2
        L.or_get_ring_f64.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.or_constants64.argtypes = [P(OrParams), P(OrConsts64)]
        L.or_lif_update64.argtypes = [P(OrConsts64), P(OrParams), ctypes.c_uint32, P(ctypes.c_double),
                                      P(ctypes.c_double), P(ctypes.c_uint8), ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int]
        L.or_set_state.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 3
        L.or_get_stats.argtypes = [ctypes.c_void_p, u64p, u64p, u64p]
        L.or_gen_rows.argtypes = [P(OrParams), ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p]
        L.or_gen_rows_list.argtypes = [P(OrParams), ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.or_gen_rows_v.argtypes = [P(OrParams), ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.or_pair_stencil.argtypes = [P(OrParams), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_uint32, u32p]
        L.or_weight_table.argtypes = [P(OrParams), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.or_delay_table.argtypes = [P(OrParams), ctypes.c_void_p, u32p]
        L.or_get_row_ptr.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.or_initial_V.argtypes = [P(OrParams), ctypes.c_uint32]
        L.or_initial_V.restype = ctypes.c_float
        L.or_drive.argtypes = [P(OrParams), P(OrConsts), ctypes.c_uint32, ctypes.c_uint32, u32p,
                               P(ctypes.c_int)]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key):
    """Philox4x32-10 of one 128-bit counter under a 64-bit key (as 2 words)."""
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox(c, k, o)
    return [int(x) for x in o]


def bf16_bits(w: float) -> int:
    return int(lib().or_bf16_bits(ctypes.c_float(w)))


def constants(cfg: dict) -> dict:
    p = params(cfg)
    c = OrConsts()
    if lib().or_constants(ctypes.byref(p), ctypes.byref(c)):
        raise ValueError(lib().or_error().decode())
    out = {f[0]: getattr(c, f[0]) for f in OrConsts._fields_ if f[0] != "pois"}
    out["pois"] = [int(c.pois[k]) for k in range(c.pois_len)]
    return out


def cdf_table(cfg: dict, module: int):
    """(thresholds uint32, target modules, FP64 normalised kernel values) of one source module."""
    p = params(cfg)
    cap = 4096
    T = np.zeros(cap, np.uint32)
    TM = np.zeros(cap, np.uint32)
    pr = np.zeros(cap, np.float64)
    n = ctypes.c_uint32()
    r = lib().or_cdf_table(ctypes.byref(p), module,
                           T.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                           TM.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                           pr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cap, ctypes.byref(n))
    if r:
        raise ValueError(lib().or_error().decode())
    k = n.value
    return T[:k].copy(), TM[:k].copy(), pr[:k].copy()


def lif_update(cfg: dict, V: float, c: float, ref: int, exc: bool, I_fx: int, forced=False):
    """One neuron update; returns (V, c, ref, spiked)."""
    p = params(cfg)
    k = OrConsts()
    if lib().or_constants(ctypes.byref(p), ctypes.byref(k)):
        raise ValueError(lib().or_error().decode())
    v = ctypes.c_float(V)
    cf = ctypes.c_float(c)
    r = ctypes.c_uint8(ref)
    s = lib().or_lif_update(ctypes.byref(k), ctypes.byref(p), ctypes.byref(v), ctypes.byref(cf),
                            ctypes.byref(r), int(bool(exc)), int(I_fx), int(bool(forced)))
    return v.value, cf.value, r.value, bool(s)


def constants64(cfg: dict) -> dict:
    """The FP64 mode's propagator constants a_m, a_c, kc (double)."""
    k = OrConsts64()
    if lib().or_constants64(ctypes.byref(params(cfg)), ctypes.byref(k)):
        raise ValueError(lib().or_error().decode())
    return {"a_m": k.a_m, "a_c": k.a_c, "kc": k.kc}


def lif_update64(cfg: dict, V: float, c: float, ref: int, exc: bool, I_mV: float, forced=False):
    """One neuron update of the FP64 mode (input in mV); returns (V, c, ref, spiked)."""
    p = params(cfg)
    k = OrConsts64()
    if lib().or_constants64(ctypes.byref(p), ctypes.byref(k)):
        raise ValueError(lib().or_error().decode())
    ref_steps = constants(cfg)["ref_steps"]
    v = ctypes.c_double(V)
    cd = ctypes.c_double(c)
    r = ctypes.c_uint8(ref)
    s = lib().or_lif_update64(ctypes.byref(k), ctypes.byref(p), ref_steps, ctypes.byref(v), ctypes.byref(cd),
                              ctypes.byref(r), int(bool(exc)), float(I_mV), int(bool(forced)))
    return v.value, cd.value, r.value, bool(s)


def gen_rows(cfg: dict, first: int, count: int):
    """Synapse rows [first, first + count) without building the whole network."""
    p = params(cfg)
    K = int(cfg["K"])
    tgt = np.empty(count * K, np.uint32)
    w = np.empty(count * K, np.float32)
    d = np.empty(count * K, np.uint8)
    if lib().or_gen_rows(ctypes.byref(p), first, count, _ptr(tgt), _ptr(w), _ptr(d)):
        raise ValueError(lib().or_error().decode())
    return tgt, w, d


def gen_rows_v(cfg: dict, first: int, count: int):
    """Rows [first, first + count) of either connection rule, back to back:
    (targets, weights, delays, row lengths)."""
    p = params(cfg)
    c = constants(cfg)
    M = int(cfg["neurons_per_module"])
    per_row = int(cfg.get("K", 0)) if int(p.conn_rule) == 0 else max(1, c["n_pair_offsets"]) * M
    cap = max(1, per_row * count)
    tgt = np.empty(cap, np.uint32)
    w = np.empty(cap, np.float32)
    d = np.empty(cap, np.uint8)
    ln = np.empty(max(1, count), np.uint32)
    if lib().or_gen_rows_v(ctypes.byref(p), first, count, cap, _ptr(tgt), _ptr(w), _ptr(d), _ptr(ln)):
        raise ValueError(lib().or_error().decode())
    n = int(ln[:count].sum())
    return tgt[:n].copy(), w[:n].copy(), d[:n].copy(), ln[:count].copy()


def gen_rows_list(cfg: dict, ids):
    """Rows of the neurons `ids` (any order, either rule), back to back:
    (targets, weights, delays, row lengths)."""
    ids = np.ascontiguousarray(ids, np.uint32)
    p = params(cfg)
    c = constants(cfg)
    M = int(cfg["neurons_per_module"])
    per_row = int(cfg.get("K", 0)) if int(p.conn_rule) == 0 else max(1, c["n_pair_offsets"]) * M
    cap = max(1, per_row * len(ids))
    tgt = np.empty(cap, np.uint32)
    w = np.empty(cap, np.float32)
    d = np.empty(cap, np.uint8)
    ln = np.empty(max(1, len(ids)), np.uint32)
    if lib().or_gen_rows_list(ctypes.byref(p), _ptr(ids), len(ids), cap, _ptr(tgt), _ptr(w), _ptr(d), _ptr(ln)):
        raise ValueError(lib().or_error().decode())
    n = int(ln[:len(ids)].sum())
    return tgt[:n], w[:n], d[:n], ln[:len(ids)].copy()


def pair_stencil(cfg: dict):
    """(dx, dy, probability, uint64 threshold) of the per-pair law's stencil."""
    p = params(cfg)
    n = ctypes.c_uint32()
    if lib().or_pair_stencil(ctypes.byref(p), None, None, None, None, 0, ctypes.byref(n)):
        raise ValueError(lib().or_error().decode())
    k = n.value
    dx = np.empty(k, np.int32)
    dy = np.empty(k, np.int32)
    pr = np.empty(k, np.float64)
    th = np.empty(k, np.uint64)
    lib().or_pair_stencil(ctypes.byref(p), _ptr(dx), _ptr(dy), _ptr(pr), _ptr(th), k, ctypes.byref(n))
    return dx, dy, pr, th


def weight_table(cfg: dict, exc: bool):
    """(float32, float64) 4096-entry Gaussian efficacy table."""
    tab = np.empty(4096, np.float32)
    tab64 = np.empty(4096, np.float64)
    lib().or_weight_table(ctypes.byref(params(cfg)), 1 if exc else 0, _ptr(tab), _ptr(tab64))
    return tab, tab64


def delay_table(cfg: dict):
    """Thresholds of the exponential delay law (uint64)."""
    thr = np.empty(256, np.uint64)
    n = ctypes.c_uint32()
    if lib().or_delay_table(ctypes.byref(params(cfg)), _ptr(thr), ctypes.byref(n)):
        raise ValueError(lib().or_error().decode())
    return thr[:n.value].copy()


def initial_V(cfg: dict, i: int) -> float:
    return float(lib().or_initial_V(ctypes.byref(params(cfg)), i))


def drive(cfg: dict, i: int, t: int):
    """(external count, forced flag) of neuron i at step t."""
    p = params(cfg)
    k = OrConsts()
    lib().or_constants(ctypes.byref(p), ctypes.byref(k))
    n = ctypes.c_uint32()
    f = ctypes.c_int()
    lib().or_drive(ctypes.byref(p), ctypes.byref(k), i, t, ctypes.byref(n), ctypes.byref(f))
    return int(n.value), bool(f.value)


def poisson_count(cfg: dict, u0: int) -> int:
    p = params(cfg)
    k = OrConsts()
    lib().or_constants(ctypes.byref(p), ctypes.byref(k))
    return int(lib().or_poisson_count(ctypes.byref(k), u0))


class OracleNet:
    """One simulated network, built and stepped by the oracle."""

    def __init__(self, cfg: dict, fp64: bool = False):
        self.cfg = dict(cfg)
        self._p = params(cfg)
        self.consts = constants(cfg)
        self.fp64 = fp64
        self._h = lib().or_create(ctypes.byref(self._p), 1 if fp64 else 0)
        if not self._h:
            raise ValueError(lib().or_error().decode())
        self.N = self.consts["N"]
        self.K = int(cfg.get("K", 0))
        self.D = self.consts["D"]

    def close(self):
        if self._h:
            lib().or_destroy(self._h)
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

    @property
    def t(self) -> int:
        return int(lib().or_time(self._h))

    def step(self, n: int = 1):
        if lib().or_step(self._h, int(n)):
            raise RuntimeError(lib().or_error().decode())

    def set_delivery_shuffle(self, seed: int):
        lib().or_set_delivery_shuffle(self._h, seed)

    def csr(self):
        ns = int(lib().or_n_synapses(self._h))
        tgt = np.empty(ns, np.uint32)
        d = np.empty(ns, np.uint8)
        if self.fp64:
            w = np.empty(ns, np.float64)
            lib().or_get_csr(self._h, _ptr(tgt), None, _ptr(d))
            lib().or_get_csr_f64(self._h, _ptr(w))
        else:
            w = np.empty(ns, np.float32)
            lib().or_get_csr(self._h, _ptr(tgt), _ptr(w), _ptr(d))
        return tgt, w, d

    def row_ptr(self):
        rp = np.empty(self.N + 1, np.uint64)
        lib().or_get_row_ptr(self._h, _ptr(rp))
        return rp

    def raster(self):
        n = int(lib().or_raster_size(self._h))
        st = np.empty(n, np.uint32)
        ids = np.empty(n, np.uint32)
        if n:
            lib().or_get_raster(self._h, _ptr(st), _ptr(ids))
        return st, ids

    def clear_raster(self):
        lib().or_clear_raster(self._h)

    def state(self):
        N, D = self.N, self.D
        ref = np.empty(N, np.uint8)
        if self.fp64:
            V = np.empty(N, np.float64)
            c = np.empty(N, np.float64)
            ring = np.empty(D * N, np.float64)
            lib().or_get_state(self._h, None, None, _ptr(ref), None)
            lib().or_get_state_f64(self._h, _ptr(V), _ptr(c))
            lib().or_get_ring_f64(self._h, _ptr(ring))
            return {"V": V, "c": c, "ref": ref, "ring": ring.reshape(D, N)}
        V = np.empty(N, np.float32)
        c = np.empty(N, np.float32)
        ring = np.empty(D * N, np.int32)
        lib().or_get_state(self._h, _ptr(V), _ptr(c), _ptr(ref), _ptr(ring))
        return {"V": V, "c": c, "ref": ref, "ring": ring.reshape(D, N)}

    def set_state(self, V=None, c=None, ref=None):
        dt = np.float64 if self.fp64 else np.float32
        V = None if V is None else np.ascontiguousarray(V, dt)
        c = None if c is None else np.ascontiguousarray(c, dt)
        ref = None if ref is None else np.ascontiguousarray(ref, np.uint8)
        if self.fp64:
            lib().or_set_state_f64(self._h, _ptr(V), _ptr(c))
            lib().or_set_state(self._h, None, None, _ptr(ref))
        else:
            lib().or_set_state(self._h, _ptr(V), _ptr(c), _ptr(ref))

    def stdp(self):
        """(accumulated change of every synapse in 2^-16 mV, post trace y, pre trace x)."""
        ns = int(lib().or_n_synapses(self._h))
        delta = np.zeros(ns, np.int64)
        y = np.empty(self.N, np.float32)
        x = np.empty(self.N, np.float32)
        lib().or_get_stdp(self._h, _ptr(delta), _ptr(y), _ptr(x))
        return delta, y, x

    def stats(self):
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        lib().or_get_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return {"spikes": a.value, "rec_events": b.value, "ext_events": c.value}
