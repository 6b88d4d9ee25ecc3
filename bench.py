"""Benchmark of the per-timestep hot path: synaptic events per second on one GB300.

Workload: the 24x24-module Gaussian network (720,000 LIF-SFA neurons, K = 1,125,
810 M synapses, FP32 weights), spiking at the paper's Gaussian rate of 7.5 Hz
(imposed Bernoulli spikes on top of the model's own dynamics, whose specified
drive alone leaves the network nearly silent).  One benchmark step = 1,000
simulated 1 ms time steps (one simulated second): for every time step the fused
neuron kernel and the delivery kernel, through the C ABI.  The synapse table
(6.5 GB: a 32-bit target | delay word and an f32 weight per synapse) is far
larger than L2, so every step streams it from HBM.

value       recurrent synaptic events / s (events = spikes x out-degree, from the
            device counters), device-timed with CUDA events over K steps.
e2e         the same metric for whole jobs through the public API: build the
            network from the host description, simulate 10,000 steps reading
            the raster into pinned host memory every 1,000 steps, destroy.
roofline    the persistent kernel: algorithmic bytes (8 B per recurrent event:
            one 32-bit target | delay word + f32 weight; 8 B per neuron and
            step: its ring slot read and cleared, the neuron state staying on
            chip through a launch) / its CUDA-event time, against the
            measured HBM copy bandwidth.
cpu_baseline  the oracle (single-threaded C) on a bounded sample of the same
            model, simulation phase only, like `value`.

--impl reference runs the oracle arm on the host cores (this project's
reference is the CPU oracle; the paper's own simulator is not available).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "synaptic events/s on 1 GB300, % of HBM roofline; served p50/p99 latency"
UNIT = "synaptic events/s"
# algorithmic bytes of the method: per recurrent event the synapse's uint32
# target, weight (f32 / bf16) and uint8 delay; per neuron and step its input
# slot read and cleared (4 + 4), V and c read and written (16), ref (2)
ALG_BYTES_PER_EVENT = {"f32": 9, "bf16": 7}
ALG_NEURON_BYTES = 26
# what this build's table layout moves: one 32-bit target | delay << 24 word
# and the weight
BYTES_PER_EVENT = {"f32": 8, "bf16": 6}
# neuron update, schedule 2: the ring slot read and cleared; V, c (f32) and ref
# (u8) stay in shared memory for the whole launch (read and written back once
# per launch).  Schedules 4 and 5: the state is read and written every step (18 B)
# and one ring row is read and cleared (8 B).
NEURON_BYTES = {2: 2 * 4, 3: 2 * 4 + 18, 4: 18 + 8, 5: 18 + 8}
# random 4-byte red.global.add.s32 into an L2-resident buffer (4-60 MB), measured on
# GB300 by `bench.py --calibrate`: the rate that bounds the push delivery, one
# reduction per recurrent synaptic event
L2_RED_PER_S = 2.2e11
TIMESTEPS_PER_STEP = 1000
JOB_TIMESTEPS = 10000

# DRAM bytes (read + write) of the persistent kernel per recurrent event, from
# one ncu capture of a smaller case of the same model, valid only for the
# kernel sources it was taken on.
NCU_TRAFFIC = {
    2: {"kernel": "k_run_steps", "source_sha256": "b90c0415b662555f7b21f9ac18d86c85151df74431e875411f5be0250ca31c09",
        "bytes_per_event": 8.39,
        "capture": "ncu --set full, 12x12 Gaussian patch (180,000 neurons, K=1125), one 30-step launch: "
                   "376.9 MB DRAM read+write for 44.9 M recurrent events, scaled to a launch by its events"},
    5: {"kernel": "k_run_steps_pull", "source_sha256": "21c6397f6a2eddcc4eed07e53a1a027d1d2cb080cccc1dbcfce389a977c85ae5",
        "bytes_per_event": 9.31,
        "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum, 16x16 Gaussian patch (320,000 "
                   "neurons, K=1125, module-aligned bands as at 24x24), one 300-step launch: 7,486.9 MB DRAM "
                   "read+write for 804.0 M recurrent events (a 30-step launch: 819.5 MB for 81.2 M, so ~70 MB "
                   "per launch are fixed -- the window filled from and returned to the ring -- and 9.22 B per "
                   "event), scaled to a launch by its events"},
}
KERNEL_SOURCES = {2: "persistent_kernels.cu", 5: "persistent_pull.cu"}


def _log(*a):
    print(*a, file=sys.stderr, flush=True)


def _kernel_source_sha(schedule=2):
    """Hash of every source the persistent kernel of `schedule` is compiled from."""
    h = hashlib.sha256()
    for f in (KERNEL_SOURCES[schedule], "device_common.cuh", "grid_common.cuh", "philox.cuh", "snn_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1803_08833_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), "snn_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local, dist


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _reduce(dist, value, op):
    if dist is None:
        return value
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def workload(seed=1, grid=24, K=None, layout="draw"):
    from paper_1803_08833_gb300 import workloads as W
    cfg = W.gauss_24x24_k1125(seed=seed, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ, table_layout=layout)
    if K is not None:
        cfg["K"] = K
    return W.patch(cfg, grid) if grid != 24 else cfg


def config_block(cfg, extra=None):
    g = cfg["grid_w"]
    n = g * g * cfg["neurons_per_module"]
    d = {
        "workload": "gauss_%dx%d_k1125: %dx%d modules x 1250 LIF-SFA neurons (%s), K=1125 "
                    "(%dM synapses), Gaussian sigma=100um cut at 3 sigma, FP32 weights, dt=1 ms"
                    % (g, g, g, g, format(n, ","), round(n * 1125 / 1e6)),
        "imposed_rate_hz": cfg["imposed_rate_hz"],
        "ext_drive": "%.0f Hz x %.1f mV Poisson" % (cfg["ext_rate_hz"], cfg["J_ext_mV"]),
        "l2": "inputs larger than L2 (129 MB): the %.1f GB synapse table (8 B per synapse, rows padded to "
              "1128) is streamed every step" % (n * 1128 * 8 / 1e9),
        "parallelism": "replicas",
    }
    if extra:
        d.update(extra)
    return d


# CPU part numbers of the Arm implementer (0x41) as /proc/cpuinfo reports them
_ARM_PARTS = {0xd0c: "Neoverse-N1", 0xd40: "Neoverse-V1", 0xd49: "Neoverse-N2", 0xd4f: "Neoverse-V2",
              0xd8e: "Neoverse-N3", 0xd84: "Neoverse-V3"}


def host_cpu():
    """The host the CPU baseline ran on: architecture, logical CPUs and model
    (lscpu's model name, else /proc/cpuinfo's model name or Arm part number)."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        impl = part = None
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    key, _, val = line.partition(":")
                    key, val = key.strip().lower(), val.strip()
                    if key in ("model name", "cpu model") and val:
                        model = val
                        break
                    if key == "cpu implementer" and impl is None:
                        impl = val
                    if key == "cpu part" and part is None:
                        part = val
        except OSError:
            pass
        if not model and impl and part:
            try:
                model = _ARM_PARTS.get(int(part, 16), "part %s" % part) if int(impl, 16) == 0x41 else \
                    "implementer %s part %s" % (impl, part)
            except ValueError:
                model = "implementer %s part %s" % (impl, part)
    return {"arch": platform.machine(), "logical_cpus": os.cpu_count(), "model": model}


# --------------------------------------------------------------------------
ORACLE_SETTLE_STEPS = 100  # simulated steps run before any oracle timing


def oracle_sample_desc(cfg, settle, timed_steps, build_s):
    n = cfg["grid_w"] * cfg["grid_h"] * cfg["neurons_per_module"]
    return ("oracle (single-threaded C) on the full workload network (%d neurons, K=%d, imposed %.1f Hz): built "
            "once (%.0f s, not timed), %d settling steps, then %d simulated 1 ms steps timed (a truncated window of "
            "the 1,000-step bench step; recurrent events / window time), simulation phase only"
            % (n, cfg["K"], cfg["imposed_rate_hz"], build_s, settle, timed_steps))


def cpu_oracle_full(cfg, window_steps, settle=ORACLE_SETTLE_STEPS):
    """Oracle simulation-phase throughput on the full benchmark network."""
    import oracle
    t0 = time.perf_counter()
    net = oracle.OracleNet(cfg)
    build_s = time.perf_counter() - t0
    net.step(settle)
    s0 = net.stats()
    t0 = time.perf_counter()
    net.step(window_steps)
    dt = time.perf_counter() - t0
    ev = net.stats()["rec_events"] - s0["rec_events"]
    net.close()
    return {"value": ev / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": oracle_sample_desc(cfg, settle, window_steps, build_s), "host": host_cpu(),
            "window_steps": window_steps, "window_s": dt, "events": ev, "build_s": build_s}


def run_reference(args):
    rank, ws, local, dist = _dist()
    if rank != 0:
        return 0
    cfg = workload(grid=args.grid)
    import oracle
    steps_per = args.ref_sample_steps
    settle = ORACLE_SETTLE_STEPS if args.ref_settle_steps is None else args.ref_settle_steps
    t0 = time.perf_counter()
    net = oracle.OracleNet(cfg)
    build_s = time.perf_counter() - t0
    net.step(settle)
    for _ in range(args.warmup):
        net.step(steps_per)
    s0 = net.stats()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        net.step(steps_per)
    dt = time.perf_counter() - t0
    s1 = net.stats()
    net.close()
    value = (s1["rec_events"] - s0["rec_events"]) / dt
    desc = oracle_sample_desc(cfg, settle + args.warmup * steps_per, args.steps * steps_per, build_s)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1000.0 / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config_block(cfg),
        "detail": {"sample": desc, "timesteps_per_step": steps_per,
                   "note": "each bench step is a bounded sample of %d simulated steps of the same network; the "
                           "metric is per event, so it compares with the GPU arm's 1,000-step bench steps"
                           % steps_per},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _cpu_baseline_child(cfg, window_steps, q):
    q.put(cpu_oracle_full(cfg, window_steps))


# --------------------------------------------------------------------------
def run_gpu(args):
    rank, ws, local, dist = _dist()
    import numpy as np
    import torch

    from paper_1803_08833_gb300 import _build, snn

    if rank == 0 or dist is None:
        _build.build()
    _barrier(dist)
    torch.cuda.set_device(local)
    schedule = 5 if args.schedule is None else args.schedule
    cfg = workload(seed=1 + rank, grid=args.grid, K=args.K, layout="grouped" if schedule in (3, 5) else "draw")
    T = args.timesteps
    peak, peak_kind = _peaks()
    stream = torch.cuda.current_stream()

    # the CPU baseline (the oracle on the same network, one core) runs in a
    # spawned process beside the GPU legs
    cpu_proc = cpu_q = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        cpu_q = ctx.Queue()
        cpu_proc = ctx.Process(target=_cpu_baseline_child, args=(cfg, args.cpu_window, cpu_q), daemon=True)
        cpu_proc.start()

    t_build = time.perf_counter()
    net = snn.Network(cfg, raster_capacity=T * 20000)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t_build
    try:
        net.set_schedule(schedule, args.block)
    except snn.SnnError as e:
        if args.schedule is not None:
            raise
        # the default pulled windows need a window row of each SM's band in shared memory
        # (up to ~50,000 neurons per SM on a GB300); larger networks run the push kernel
        _log("schedule 5 unavailable here (%s); using schedule 2" % e)
        schedule = 2
        net.set_schedule(schedule, args.block)
    net.set_timing(args.timing_every)

    for _ in range(args.warmup):
        net.step(T)
        net.clear_raster()
    torch.cuda.synchronize()
    kt0 = net.kernel_time()
    s0 = net.stats()
    l0 = snn.launch_count()

    ev_a = torch.cuda.Event(enable_timing=True)
    ev_b = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        _barrier(dist)
        torch.cuda.synchronize()
        ev_a.record(stream)
        for _ in range(args.steps):
            net.step(T)
            net.clear_raster()
        ev_b.record(stream)
        torch.cuda.synchronize()
        _barrier(dist)
    launches = snn.launch_count() - l0
    ms = ev_a.elapsed_time(ev_b)
    s1 = net.stats()
    kt1 = net.kernel_time()
    rec = s1["rec_events"] - s0["rec_events"]
    ext = s1["ext_events"] - s0["ext_events"]
    spikes = s1["n_spikes"] - s0["n_spikes"]

    ms_max = _reduce(dist, ms, _max_op(dist))
    rec_all = _reduce(dist, rec, _sum_op(dist))
    value = rec_all / (ms_max / 1000.0)

    dl = kt1["deliver_launches"] - kt0["deliver_launches"]
    dms = kt1["deliver_ms"] - kt0["deliver_ms"]
    nms = kt1["neuron_ms"] - kt0["neuron_ms"]
    pl = kt1["persistent_launches"] - kt0["persistent_launches"]
    pms = kt1["persistent_ms"] - kt0["persistent_ms"]
    # algorithmic bytes of the dominant kernel per launch / its mean CUDA-event duration
    steps_timed = args.steps * T
    traffic = None
    packed = None
    if pl > 0:  # persistent schedule: one launch = T steps of neuron update + delivery
        kname = {3: "k_run_steps_tiled", 4: "k_run_steps_owned", 5: "k_run_steps_pull"}.get(schedule, "k_run_steps")
        kernel = "%s<f32> (persistent: neuron update + delivery, %d steps per launch)" % (kname, T)
        launches_timed = pl
        launch_s = pms / pl / 1000.0
        alg_per_launch = (ALG_BYTES_PER_EVENT["f32"] * rec + ALG_NEURON_BYTES * net.N * steps_timed) / max(args.steps, 1)
        achieved = alg_per_launch / launch_s / 1e9 if pms > 0 else None
        bytes_note = ("%d B per recurrent event (uint32 target + f32 weight + uint8 delay) + %d B per neuron per "
                      "step" % (ALG_BYTES_PER_EVENT["f32"], ALG_NEURON_BYTES))
        nb = NEURON_BYTES.get(schedule, NEURON_BYTES[2])
        pk = (BYTES_PER_EVENT["f32"] * rec + nb * net.N * steps_timed) / max(args.steps, 1)
        packed = {"achieved": pk / launch_s / 1e9 if pms > 0 else None,
                  "frac": pk / launch_s / 1e9 / peak if pms > 0 else None,
                  "bytes_per_launch": pk,
                  "bytes": "%d B per recurrent event (target | delay word + f32 weight) + %d B per neuron per step "
                           "(what this schedule moves)" % (BYTES_PER_EVENT["f32"], nb)}
        nt = NCU_TRAFFIC.get(schedule)
        if nt and nt["bytes_per_event"] and nt["source_sha256"] == _kernel_source_sha(schedule):
            traffic = nt["bytes_per_event"] * rec / max(args.steps, 1)
    else:
        kernel = "k_deliver_warp<f32>"
        launches_timed = dl
        alg_per_launch = ALG_BYTES_PER_EVENT["f32"] * rec / steps_timed
        achieved = alg_per_launch / (dms / max(dl, 1) / 1000.0) / 1e9 if dms > 0 else None
        bytes_note = "%d B per recurrent event" % ALG_BYTES_PER_EVENT["f32"]
    dphase_s = (s1["deliver_phase_ns"] - s0["deliver_phase_ns"]) / 1e9 if pl else 0.0
    delivery_phase = ({"achieved": ALG_BYTES_PER_EVENT["f32"] * rec / dphase_s / 1e9,
                       "frac": ALG_BYTES_PER_EVENT["f32"] * rec / dphase_s / 1e9 / peak,
                       "bytes": "%d B per recurrent event over the delivery phases (GPU timer of CTA 0, their "
                                "barriers included)" % ALG_BYTES_PER_EVENT["f32"]} if dphase_s > 0 else None)
    net.set_timing(0)

    # end-to-end jobs through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(snn, cfg, args.e2e_jobs, stream, schedule)
    net.close()

    batched = None if args.no_batched else run_batched(snn, args, stream)
    precision = None if args.no_precision else run_precision(snn, args, stream)
    table_one = None if args.no_table_one else run_table_one(snn, args, stream)
    served = None if args.no_served else run_served(snn, args, stream)

    cpu = None
    if cpu_proc is not None:
        try:
            cpu = cpu_q.get(timeout=1800)
        except Exception as e:  # report, never hang the bench
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": repr(e)}
        cpu_proc.join(timeout=60)

    if rank != 0:
        return 0
    ck = clocks.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_block(cfg),
        "detail": dict({"build_ms": round(t_build * 1000.0, 1),
                                     "timesteps_per_step": T,
                                     "spikes_per_timestep": spikes / (args.steps * T),
                                     "rate_hz": spikes / (args.steps * T) / net.N * 1000.0,
                                     "equivalent_events_per_s": (rec + ext) / (ms / 1000.0),
                                     "schedule": schedule,
                                     "table_layout": cfg["table_layout"],
                                     "neuron_kernel_us": 1000.0 * nms / max(dl, 1) if dl else None,
                                     "deliver_kernel_us": 1000.0 * dms / max(dl, 1) if dl else None,
                                     "persistent_us_per_step": 1000.0 * pms / steps_timed if pl else None,
                                     "neuron_phase_us": (s1["neuron_phase_ns"] - s0["neuron_phase_ns"]) / 1e3 / steps_timed
                                     if pl else None,
                                     "deliver_phase_us": (s1["deliver_phase_ns"] - s0["deliver_phase_ns"]) / 1e3 / steps_timed
                                     if pl else None,
                                     # one L2 reduction per recurrent event: the reduction rate of the
                                     # delivery phase (its barrier included), against ~2.2e11/s measured
                                     # for random reductions alone (bench.py --calibrate)
                                     "delivery_phase_l2_reductions_per_s":
                                     rec / ((s1["deliver_phase_ns"] - s0["deliver_phase_ns"]) / 1e9)
                                     if pl and s1["deliver_phase_ns"] > s0["deliver_phase_ns"] else None,
                                     "kernel_timing": ("CUDA events around every persistent launch of the timed "
                                                       "region; phases from the GPU timer of CTA 0" if pl else
                                                       "CUDA events around the kernels of every %d-th simulated "
                                                       "step of the timed region" % args.timing_every)}),
        "roofline": {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "algorithmic_bytes": bytes_note, "bytes_per_launch": alg_per_launch,
                     "packed": packed, "delivery_phase": delivery_phase,
                     "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured"
                     else "fallback 6.8 TB/s",
                     "launches_timed": launches_timed},
        # the bound that actually limits the path: one random L2 reduction per event
        "l2_reduction_bound": {"achieved": rec / (pms / 1000.0) if pl and pms > 0 else None,
                               "peak": L2_RED_PER_S, "unit": "reductions/s",
                               "frac": rec / (pms / 1000.0) / L2_RED_PER_S if pl and pms > 0 else None,
                               "peak_source": "calibrated (bench.py --calibrate): random red.global.add.s32 "
                                              "into a 4-60 MB buffer",
                               "note": "whole persistent launch (neuron phase, barriers and scan included)"
                                       + ("; schedule 5 reduces in L2 only the events of delay > W, the rest "
                                          "go to shared memory, so this bound does not cap it" if schedule == 5
                                          else "")},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "batched": batched,
        "served": served,
        "precision": precision,
        "table_one": table_one,
        "gpu_launches": launches,
        "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_e2e(snn, cfg, jobs, stream, schedule):
    """Whole jobs through the public API: build from the host description,
    simulate JOB_TIMESTEPS reading the raster into pinned host memory after
    every 1,000 steps, destroy.  Device-side inputs are never reused."""
    import ctypes

    import numpy as np
    import torch
    cap = TIMESTEPS_PER_STEP * 20000
    h_steps = torch.empty(cap, dtype=torch.int32, pin_memory=True)
    h_ids = torch.empty(cap, dtype=torch.int32, pin_memory=True)
    a_steps = h_steps.numpy().view(np.uint32)
    a_ids = h_ids.numpy().view(np.uint32)
    total_ev, total_t, d2h = 0, 0.0, 0
    for j in range(jobs + 1):  # the first job warms the allocator and is not counted
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net = snn.Network(dict(cfg, seed=100 + j), raster_capacity=cap, stream=stream)
        net.set_schedule(schedule)
        got = 0
        for _ in range(JOB_TIMESTEPS // TIMESTEPS_PER_STEP):
            net.step(TIMESTEPS_PER_STEP)
            got += net.read_spikes_into(a_steps, a_ids)
            net.clear_raster()
        st = net.stats()
        net.close()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if j > 0:
            total_ev += st["rec_events"]
            total_t += dt
            d2h += got * 8 + ctypes.sizeof(snn.SnnStats)
    h2d = ctypes.sizeof(snn.SnnConfig)
    return {"value": total_ev / total_t, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": int(d2h / max(jobs, 1)),
            "step": "one job: build + %d timesteps + raster readout every %d steps" % (JOB_TIMESTEPS,
                                                                                       TIMESTEPS_PER_STEP),
            "jobs": jobs}


def run_batched(snn, args, stream):
    """64 independent instances (grid side 4..16, Gaussian or exponential,
    f32 or bf16) advanced 2,000 steps in one persistent launch, against the
    same instances run one per launch (each its own persistent launch)."""
    import torch
    from paper_1803_08833_gb300 import workloads as W
    inst = W.batched_instances(n=args.batch_n, steps=args.batch_steps)
    nets = [snn.Network(c, raster_capacity=1) for c, _ in inst]
    for n in nets:
        n.set_schedule(2)
    steps = [s for _, s in inst]

    def events():
        return sum(n.stats()["rec_events"] for n in nets)

    def timed_batch(batch):
        batch.step([20] * len(nets))  # warm-up (captures the graph, measures the groups)
        torch.cuda.synchronize()
        e0, l0 = events(), snn.launch_count()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        batch.step(steps)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), events() - e0, snn.launch_count() - l0

    with snn.Batch(nets, stream=stream) as batch:
        batch.set_graph(True)
        # the fixed default: grouped layout, launch shape 0, half the L2 per wave
        ms_fixed, ev_fixed, _ = timed_batch(batch)
        # the same waves in one global neuron / task space each
        batch.set_mode("global")
        ms_global, ev_global, _ = timed_batch(batch)
        # the autotuned layout, shape and ring budget (tuning restores every state)
        tuned = batch.autotune(trial_steps=args.batch_tune_steps)
        ms_batched, ev_batched, launches_batched = timed_batch(batch)
        waves, ring_budget = batch.waves()
        cta = batch.groups()
    # plain: one instance per launch, back to back on the same stream
    e0 = events()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for n, s in zip(nets, steps):
        n.step(s)
    b.record(stream)
    torch.cuda.synchronize()
    ms_plain = a.elapsed_time(b)
    ev_plain = events() - e0
    neurons = sum(n.N for n in nets)
    for n in nets:
        n.close()
    v_b = ev_batched / (ms_batched / 1e3)
    v_p = ev_plain / (ms_plain / 1e3)
    v_g = ev_global / (ms_global / 1e3)
    v_f = ev_fixed / (ms_fixed / 1e3)
    return {"value": v_b, "unit": UNIT, "plain_value": v_p, "speedup_vs_plain": v_b / v_p,
            "global_value": v_g, "speedup_vs_global": v_b / v_g,
            "fixed_value": v_f, "speedup_vs_fixed": v_b / v_f,
            "tuned": {"mode": tuned["mode"], "shape": tuned["shape"], "ring_budget_mb": tuned["ring_budget"] / 2 ** 20,
                      "trial_ms_per_step": tuned["ms_per_step"], "trial_steps": args.batch_tune_steps,
                      "sweep_ms_per_step": tuned["sweep_ms_per_step"],
                      "candidates": "layout {groups, global} x shape {2 CTAs/SM x 4 tasks, 1 x 6} x ring "
                                    "budget {0.35, 0.5, 0.65} of L2, distinct wave plans only"},
            "instances": len(inst), "neurons": neurons, "steps_each": args.batch_steps,
            "ms_batched": ms_batched, "ms_global": ms_global, "ms_plain": ms_plain, "launches": launches_batched,
            "waves": waves, "ring_budget_mb": ring_budget / 2 ** 20,
            "ctas_per_instance": {"min": min(cta), "max": max(cta)},
            "workload": "64 instances, grid side U{4..16} x 1250 neurons, K=1125, Gaussian (even seed, 7.5 Hz) / "
                        "exponential (odd seed, 35 Hz), bf16 weights when seed bit 1 is set, one persistent "
                        "launch per L2-sized wave of instances in the autotuned layout, launch shape and ring "
                        "budget, replayed from one CUDA graph; vs one persistent launch per instance (plain), the "
                        "fixed default (grouped, shape 0, half the L2; fixed) and the same waves in one global "
                        "neuron / task space (global)"}


def run_precision(snn, args, stream):
    """The exponential long-range network at full size (24x24 x 1250, K = 2250,
    lambda = 290 um, cut-off 1.2 mm) with bf16 and with f32 weights, 10,000 steps
    each after 500 warm-up steps, under a 5.2 kHz drive (the low-rate state:
    the specified drive leaves it silent, above ~5.8 kHz it saturates near
    280 Hz).  The FP64 comparison, which the oracle can only afford on a patch,
    is tests/test_gpu_precision.py."""
    import numpy as np
    import torch
    from paper_1803_08833_gb300 import workloads as W
    out = {}
    rates = {}
    for dt in ("bf16", "f32"):
        cfg = W.exp_24x24_k2250(seed=1, weight_dtype=dt, ext_rate_hz=5200.0)
        with snn.Network(cfg, raster_capacity=64 << 20, stream=stream) as net:
            net.set_schedule(2)
            net.step(500)
            net.clear_raster()
            s0 = net.stats()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            net.step(args.precision_steps)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            s1 = net.stats()
            _, ids = net.read_spikes(allow_overflow=True)
            rates[dt] = np.bincount(ids, minlength=net.N) / (args.precision_steps / 1000.0)
            ev = s1["rec_events"] - s0["rec_events"]
            out[dt] = {"events_per_s": ev / (ms / 1e3), "ms_per_step": ms / args.precision_steps,
                       "rate_hz": float(rates[dt].mean()), "bytes_per_synapse": BYTES_PER_EVENT[dt],
                       "table_gb": net.device_bytes / 1e9}
    M = 1250
    mod = lambda r: r.reshape(-1, M).mean(axis=1)
    out["bf16_vs_f32"] = {
        "mean_rate_rel_err": float(rates["bf16"].mean() / rates["f32"].mean() - 1.0),
        "neuron_rate_corr": float(np.corrcoef(rates["bf16"], rates["f32"])[0, 1]),
        "module_rate_corr": float(np.corrcoef(mod(rates["bf16"]), mod(rates["f32"]))[0, 1])}
    out["workload"] = ("exp_24x24_k2250: 24x24 x 1250 neurons, K=2250 (1.62 G synapses), lambda=290 um cut at 1.2 mm, "
                       "5.2 kHz x 0.2 mV drive (low-rate state), %d steps" % args.precision_steps)
    return out


def run_table_one(snn, args, stream):
    """Table I's grids: the 24x24 network under the paper's per-pair law
    (Gaussian at 7.5 Hz, exponential at 35 Hz, bf16) and the 48x48 / 96x96
    Gaussian grids with the fixed out-degree rule (grouped rows) and 48x48
    per-pair: build time, synapses, device memory, delivery bands and
    persistent-schedule throughput."""
    import time as _t

    import torch
    from paper_1803_08833_gb300 import workloads as W
    cases = [
        ("pairwise_24x24_gauss", W.pairwise(grid=24, seed=1, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ), 1000),
        ("pairwise_24x24_exp_bf16", W.pairwise(grid=24, lateral="exp", seed=1, weight_dtype="bf16",
                                               imposed_rate_hz=W.PAPER_RATE_EXP_HZ), 300),
        ("pairwise_48x48_gauss", W.pairwise(grid=48, seed=1, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ), 300),
        ("fixed_48x48_gauss_k1125", W.gauss_48x48_k1125(seed=1, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ,
                                                        table_layout="grouped"), 300),
        ("fixed_96x96_gauss_k1125", W.gauss_96x96_k1125(seed=1, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ,
                                                        table_layout="grouped"), 100),
    ]
    out = {}
    for name, cfg, steps in cases:
        steps = max(1, int(steps * args.table_one_scale))
        torch.cuda.synchronize()
        t0 = _t.perf_counter()
        with snn.Network(cfg, raster_capacity=1 << 24, stream=stream) as net:
            torch.cuda.synchronize()
            build_ms = (_t.perf_counter() - t0) * 1e3
            syn = int(net.row_lengths().astype("int64").sum())
            bands = net.set_bands(0)
            runs = {}
            for sched in (2, 5):  # the push kernel, then the pulled windows where a window row fits
                try:
                    net.set_schedule(sched)
                except snn.SnnError as e:
                    runs[sched] = {"refused": str(e).splitlines()[0][:160]}
                    continue
                window = net.set_pull_window(0) if sched == 5 else None
                net.step(20)
                s0 = net.stats()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                net.step(steps)
                b.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                s1 = net.stats()
                ev = s1["rec_events"] - s0["rec_events"]
                runs[sched] = {"us_per_step": ms * 1e3 / steps, "events_per_s": ev / (ms / 1e3),
                               "rate_hz": (s1["n_spikes"] - s0["n_spikes"]) / (net.N * steps) * 1000.0}
                if sched == 5:
                    runs[sched]["window"], runs[sched]["band_mode"] = window, net.pull_band_mode
            best = max((k for k in runs if "events_per_s" in runs[k]), key=lambda k: runs[k]["events_per_s"])
            out[name] = {"neurons": net.N, "synapses": syn, "device_gb": round(net.device_bytes / 1e9, 2), "bands": bands,
                         "build_ms": round(build_ms, 1), "steps": steps, "schedule": best,
                         "us_per_step": runs[best]["us_per_step"], "events_per_s": runs[best]["events_per_s"],
                         "rate_hz": runs[best]["rate_hz"], "by_schedule": runs}
    out["workload"] = ("Table I grids (100 um spacing, 1250 neurons per module); per-pair law: 80 % local, "
                       "A exp(-r^2/2 sigma^2) A=0.05 / A exp(-r/lambda) A=0.03 cut at 1/1000, inhibitory local only, "
                       "Gaussian efficacies, exponential delays (mean 5 ms); imposed paper rates; persistent schedules 2 (push) and 5 (pulled windows, where a window row fits), the "
                       "faster one reported")
    return out


def run_served(snn, args, stream):
    """Poisson stream of requests into the continuous-batching server."""
    import time as _t

    import numpy as np
    from paper_1803_08833_gb300 import workloads as W
    stream_reqs = W.served_stream(seconds=args.served_seconds, rate_hz=20.0, seed=7)
    budget = 150 << 30
    results = []
    # the batch layout of the ticks: the tuner's choice on a sample of the mix
    # (the first 16 requests as one batch, states restored after tuning)
    sample = [snn.Network(cfg, raster_capacity=1 << 10, stream=stream) for _, cfg, _ in stream_reqs[:16]]
    for n in sample:
        n.set_schedule(2)
    with snn.Batch(sample, stream=stream) as b:
        tuned = b.autotune(trial_steps=100)
    for n in sample:
        n.close()
    with snn.Server(budget, chunk_steps=args.served_chunk, max_slots=args.served_slots, stream=stream) as srv:
        srv.set_batch(tuned["mode"], tuned["shape"], tuned["ring_budget"])
        start = snn.now_ns()
        i = 0
        peak = 0
        while True:
            now_s = (snn.now_ns() - start) / 1e9
            while i < len(stream_reqs) and stream_reqs[i][0] <= now_s:
                t, cfg, steps = stream_reqs[i]
                srv.submit(cfg, steps, arrival_ns=start + int(t * 1e9), raster_capacity=1 << 10)
                i += 1
            a, q = srv.tick()
            peak = max(peak, a)
            results += srv.poll()
            if i == len(stream_reqs) and a == 0 and q == 0:
                break
            if a == 0 and q == 0 and i < len(stream_reqs):
                _t.sleep(max(0.0, stream_reqs[i][0] - (snn.now_ns() - start) / 1e9))
        wall = (snn.now_ns() - start) / 1e9
        st = srv.stats()
    # the same kind of requests one instance per launch (every 10th request of
    # the stream, in turn: build, persistent run, counters, destroy)
    import torch
    plain_ev, plain_s, plain_n = 0, 0.0, 0
    for t, cfg, steps in stream_reqs[::10]:
        torch.cuda.synchronize()
        t0 = snn.now_ns()
        with snn.Network(cfg, raster_capacity=1 << 10, stream=stream) as net:
            net.set_schedule(2)
            net.step(steps)
            plain_ev += net.stats()["rec_events"]
        torch.cuda.synchronize()
        plain_s += (snn.now_ns() - t0) / 1e9
        plain_n += 1
    lat = np.array([r["latency_ms"] for r in results])
    qms = np.array([r["queue_ms"] for r in results])
    ok = sum(1 for r in results if r["status"] == 0)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_queue_ms": float(qms.mean()), "requests": len(results), "ok": ok,
            "value": st["rec_events"] / wall, "unit": UNIT, "wall_s": wall, "arrival_window_s": args.served_seconds,
            "busy_value": st["rec_events"] / (st["busy_ns"] / 1e9),
            "plain_value": plain_ev / plain_s, "plain_requests": plain_n,
            "plain": "every 10th request run alone in turn (build, persistent run, destroy): events / total time",
            "gpu_busy_frac": st["busy_ns"] / 1e9 / wall, "peak_active": peak, "launches": st["launches"],
            "budget_gb": 150, "chunk_steps": args.served_chunk,
            "batch_layout": {"mode": tuned["mode"], "shape": tuned["shape"],
                             "ring_budget_mb": tuned["ring_budget"] / 2 ** 20,
                             "tuned_on": "the first 16 requests as one batch, 100 trial steps per candidate",
                             "sweep_ms_per_step": tuned["sweep_ms_per_step"]},
            "workload": "Poisson arrivals at 20 req/s (seed 7), grid side U{4..32} x 1250 neurons, K U{500..2250}, "
                        "Gaussian or exponential, every network spiking at %.1f Hz (imposed background rate), "
                        "duration U{500..5000} steps, bf16 weights, 150 GB budget, continuous batching in chunks "
                        "of %d steps" % (W.SERVED_RATE_HZ, args.served_chunk)}


def _max_op(dist):
    return None if dist is None else dist.ReduceOp.MAX


def _sum_op(dist):
    return None if dist is None else dist.ReduceOp.SUM


def run_calibration():
    """Compile and run the memory-system calibration (calibration/l2_rates.cu)."""
    from paper_1803_08833_gb300 import _build
    src = os.path.join(ROOT, "paper_1803_08833_gb300", "calibration", "l2_rates.cu")
    exe = os.path.join(_build.BUILD, "l2_rates")
    os.makedirs(_build.BUILD, exist_ok=True)
    subprocess.check_call([_build.nvcc(), *_build.ARCH, "-O3", "-o", exe, src])
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.strip()
    print(out, flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--schedule", type=int, default=None)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--e2e-jobs", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--calibrate", action="store_true", help="measure L2 reduction and stream rates, then exit")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-table-one", action="store_true")
    ap.add_argument("--table-one-scale", type=float, default=1.0, help="scale of the Table I legs' step counts")
    ap.add_argument("--precision-steps", type=int, default=10000)
    ap.add_argument("--batch-n", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=2000)
    ap.add_argument("--batch-tune-steps", type=int, default=200, help="trial steps per candidate of the batch tuner")
    ap.add_argument("--served-seconds", type=float, default=60.0)
    ap.add_argument("--served-chunk", type=int, default=250)
    ap.add_argument("--served-slots", type=int, default=64)
    ap.add_argument("--cpu-window", type=int, default=200,
                    help="simulated steps of the oracle timed on the full network for cpu_baseline")
    ap.add_argument("--ref-sample-steps", type=int, default=10,
                    help="simulated steps of the oracle per bench step in --impl reference")
    ap.add_argument("--ref-settle-steps", type=int, default=None,
                    help="untimed oracle steps before the reference arm's warm-up (default %d)" % ORACLE_SETTLE_STEPS)
    ap.add_argument("--timing-every", type=int, default=10,
                    help="time the kernels of every n-th simulated step with CUDA events")
    ap.add_argument("--grid", type=int, default=24, help="modules per side (24 = the benchmark workload)")
    ap.add_argument("--K", type=int, default=None, help="out-degree override (profiling of the neuron update only)")
    ap.add_argument("--timesteps", type=int, default=TIMESTEPS_PER_STEP, help="simulated steps per bench step")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "gb300":
        _log("note: fewer than 3 warm-up steps")
    if args.calibrate:
        return run_calibration()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
