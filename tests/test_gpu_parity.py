"""Parity of the CUDA path (through the C ABI) with the oracle.

Integer work (target tables, synapse tables, spike rasters, ring contents) must
be bit-exact; with FP32 and BF16 weights the neuron state (V, c) is bit-exact
too, because both sides evaluate the same IEEE expressions in the same order
with no fused multiply-add.
"""
import numpy as np
import pytest

import oracle
from paper_1803_08833_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    from paper_1803_08833_gb300 import _build
    from paper_1803_08833_gb300 import snn as S
    _build.build()
    S.load()
    return S


def _cdf_case(name):
    if name == "gauss4":
        return W.gauss_4x4_k1000()
    if name == "gauss24":
        return W.gauss_24x24_k1125()
    if name == "exp24":
        return W.exp_24x24_k2250()
    if name == "exp_rect":
        return dict(W.small(lateral="exp"), grid_w=13, grid_h=5)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["gauss4", "gauss24", "exp24", "exp_rect"])
def test_target_tables_equal_oracle(snn, name):
    cfg = dict(_cdf_case(name), neurons_per_module=2, K=8)  # the tables depend on the grid only
    with snn.Network(cfg) as net:
        T, TM, cnt = net.cdf()
    for m in range(cfg["grid_w"] * cfg["grid_h"]):
        oT, oTM, _ = oracle.cdf_table(cfg, m)
        n = len(oT)
        assert cnt[m] == n
        assert np.array_equal(T[m, :n], oT), m
        assert np.array_equal(TM[m, :n], oTM), m


CSR_CASES = {
    "gauss_4x4_k1000": lambda: W.gauss_4x4_k1000(seed=3),
    "ragged_k37": lambda: dict(W.small(grid=3, M=77, K=37, seed=12), grid_h=2),
    "exp_bf16": lambda: W.small(grid=6, M=50, K=203, lateral="exp", seed=4, weight_dtype="bf16"),
    "k1": lambda: W.small(grid=2, M=5, K=1, seed=2),
    "k0": lambda: W.small(grid=2, M=5, K=0, seed=2),
}


@pytest.mark.parametrize("name", sorted(CSR_CASES))
def test_synapse_table_equals_oracle(snn, name):
    cfg = CSR_CASES[name]()
    with snn.Network(cfg) as net:
        tgt, w, d = net.csr()
    ref = oracle.OracleNet(cfg)
    rt, rw, rd = ref.csr()
    assert np.array_equal(tgt, rt)
    assert np.array_equal(w.view(np.uint32), rw.view(np.uint32))
    assert np.array_equal(d, rd)


def _grouped_rows(cfg, tgt, w, d):
    """The oracle's draw-order rows, stably sorted by target module (per row)."""
    K, M = cfg["K"], cfg["neurons_per_module"]
    N = len(tgt) // K if K else 0
    tm = (tgt // M).reshape(N, K).astype(np.int64)
    order = np.argsort(tm, axis=1, kind="stable")
    take = lambda a: np.take_along_axis(a.reshape(N, K), order, axis=1).reshape(-1)
    return take(tgt), take(w), take(d)


@pytest.mark.parametrize("name", sorted(CSR_CASES))
def test_grouped_table_and_segments_equal_oracle(snn, name):
    cfg = dict(CSR_CASES[name](), table_layout="grouped")
    with snn.Network(cfg) as net:
        tgt, w, d = net.csr()
        seg = net.segments() if cfg["K"] else None
    ref = oracle.OracleNet(cfg)
    rt, rw, rd = _grouped_rows(cfg, *ref.csr())
    assert np.array_equal(tgt, rt) and np.array_equal(d, rd)
    assert np.array_equal(w.view(np.uint32), rw.view(np.uint32))
    if seg is None:
        return
    K, M = cfg["K"], cfg["neurons_per_module"]
    for i in range(0, ref.N, max(1, ref.N // 97)):
        _, TM, _ = oracle.cdf_table(cfg, i // M)
        pos = {int(m): j for j, m in enumerate(TM.tolist())}
        js = np.array([pos[int(x) // M] for x in rt[i * K:(i + 1) * K]])
        counts = np.bincount(js, minlength=len(TM))
        expect = np.concatenate([[0], np.cumsum(counts)])[:len(TM)]
        assert np.array_equal(seg[i, :len(TM)], expect), i
        assert np.all(seg[i, len(TM):] == K)


SIM_CASES = {
    # the plain 4x4 workload as specified (it falls nearly silent after the initial transient)
    "gauss4_seed1": (lambda: W.gauss_4x4_k1000(seed=1), 1000),
    "gauss4_seed2": (lambda: W.gauss_4x4_k1000(seed=2), 1000),
    "gauss4_seed3": (lambda: W.gauss_4x4_k1000(seed=3), 1000),
    # the same network at the paper's Gaussian rate (imposed) and under a stronger drive
    "gauss4_imposed7.5": (lambda: W.gauss_4x4_k1000(seed=1, imposed_rate_hz=7.5), 300),
    "gauss4_drive5k": (lambda: W.gauss_4x4_k1000(seed=2, ext_rate_hz=5000.0), 300),
    # long-range kernel, bf16 weights, the paper's exponential rate
    "exp_bf16_35hz": (lambda: W.small(grid=7, M=150, K=400, lateral="exp", seed=5, weight_dtype="bf16",
                                      imposed_rate_hz=35.0), 200),
    # ragged sizes: N not a multiple of the block, K not a multiple of the vector width
    "ragged": (lambda: dict(W.small(grid=3, M=333, K=37, seed=9, imposed_rate_hz=40.0), grid_h=2), 150),
    # adaptation and E != 0 exercised under strong drive
    "adapt_E": (lambda: W.small(grid=4, M=100, K=90, seed=6, ext_rate_hz=6000.0, E_mV=-1.5, alpha_c=0.2), 250),
}


def _compare(net, ref):
    st, ids = net.read_spikes()
    rs, ri = ref.raster()
    assert np.array_equal(st, rs) and np.array_equal(ids, ri), (len(st), len(rs))
    s, o = net.state(), ref.state()
    assert s["t"] == ref.t
    assert np.array_equal(s["V"].view(np.uint32), o["V"].view(np.uint32))
    assert np.array_equal(s["c"].view(np.uint32), o["c"].view(np.uint32))
    assert np.array_equal(s["ref"], o["ref"])
    assert np.array_equal(s["ring"], o["ring"])
    a, b = net.stats(), ref.stats()
    assert a["n_spikes"] == b["spikes"] and a["rec_events"] == b["rec_events"]
    assert a["ext_events"] == b["ext_events"]
    return len(st)


@pytest.mark.parametrize("schedule", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("name", sorted(SIM_CASES))
def test_simulation_bit_exact(snn, name, schedule):
    make, steps = SIM_CASES[name]
    cfg = make()
    if schedule in (3, 5):
        cfg["table_layout"] = "grouped"
    with snn.Network(cfg, raster_capacity=1 << 22) as net:
        net.set_schedule(schedule)
        net.step(steps)
        ref = oracle.OracleNet(cfg)
        ref.step(steps)
        n = _compare(net, ref)
    if "imposed" in name or "35hz" in name or "drive" in name:
        assert n > 1000


def test_block_sizes_agree(snn):
    cfg = W.small(grid=3, M=200, K=150, seed=3, imposed_rate_hz=50.0)
    ref = oracle.OracleNet(cfg)
    ref.step(80)
    for schedule, block in ((0, 32), (0, 128), (1, 64), (1, 256)):
        with snn.Network(cfg) as net:
            net.set_schedule(schedule, block)
            net.step(80)
            _compare(net, ref)


@pytest.mark.parametrize("schedule_b", [0, 2])
def test_steps_in_pieces_equal_one_call(snn, schedule_b):
    cfg = W.small(grid=3, M=100, K=60, seed=8, imposed_rate_hz=30.0)
    with snn.Network(cfg) as a, snn.Network(cfg) as b:
        a.step(90)
        b.set_schedule(schedule_b)
        for i, n in enumerate((1, 2, 30, 57)):
            if i == 2:
                b.set_schedule(2 - schedule_b)  # switching schedules mid-run changes nothing
            b.step(n)
        sa, sb = a.state(), b.state()
        for k in ("V", "c", "ref", "ring"):
            assert np.array_equal(sa[k], sb[k])
        assert all(np.array_equal(x, y) for x, y in zip(a.read_spikes(), b.read_spikes()))


def test_snapshot_restore_resumes_bit_exact(snn):
    cfg = W.small(grid=3, M=120, K=80, seed=14, imposed_rate_hz=25.0, ext_rate_hz=4000.0)
    with snn.Network(cfg) as a, snn.Network(cfg) as b:
        a.set_schedule(2)
        a.step(120)
        st_a, id_a = a.read_spikes()
        a.step(0)
        b.step(60)
        blob = b.snapshot()
        with snn.Network(cfg) as c:
            c.restore(blob)
            c.step(60)
            st_c, id_c = c.read_spikes()
            late = st_a >= 60
            assert np.array_equal(st_c, st_a[late]) and np.array_equal(id_c, id_a[late])
            sa, sc = a.state(), c.state()
            for k in ("V", "c", "ref", "ring", "t"):
                assert np.array_equal(sa[k], sc[k]), k
            assert c.stats()["n_spikes"] == a.stats()["n_spikes"]


def test_snapshot_of_another_network_is_rejected(snn):
    with snn.Network(W.small(seed=1)) as a, snn.Network(W.small(seed=2)) as b:
        blob = a.snapshot()
        with pytest.raises(snn.SnnError, match="different network"):
            b.restore(blob)


def test_raster_overflow_is_reported(snn):
    cfg = W.small(grid=3, M=100, K=20, seed=4, imposed_rate_hz=100.0)
    with snn.Network(cfg, raster_capacity=500) as net:
        net.step(40)
        with pytest.raises(snn.SnnError, match="SNN_EOVERFLOW"):
            net.read_spikes()
        st, ids = net.read_spikes(allow_overflow=True)
        assert len(st) == 500
        ref = oracle.OracleNet(cfg)
        ref.step(40)
        rs, ri = ref.raster()
        assert np.array_equal(st, rs[:500]) and np.array_equal(ids, ri[:500])
        assert net.stats()["n_spikes"] == len(rs)
        net.clear_raster()
        net.step(1)
        st2, _ = net.read_spikes()
        assert np.all(st2 == 40)


def test_empty_steps_and_silent_network(snn):
    cfg = W.small(grid=2, M=64, K=10, seed=1, ext_rate_hz=0.0)
    with snn.Network(cfg) as net:
        net.step(0)
        V0 = net.state()["V"]
        net.step(50)
        st, _ = net.read_spikes()
        assert len(st) == 0 and net.stats()["rec_events"] == 0
        ref = oracle.OracleNet(cfg)
        ref.step(50)
        assert np.array_equal(net.state()["V"], ref.state()["V"])
        assert V0.max() < cfg["V_th_mV"]


def _full_size_check(snn, cfg, n_rows=1500, seed=0, schedule=0):
    """At the full configuration: sampled synapse rows, the first step of sampled
    neurons, the exact ring after the first delivery, and invariants."""
    rng = np.random.default_rng(seed)
    with snn.Network(cfg, raster_capacity=1 << 24) as net:
        N, K, M = net.N, net.K, cfg["neurons_per_module"]
        rows = np.unique(np.concatenate([
            rng.integers(0, N, n_rows), [0, 1, M - 1, M, N // 2, N - 2, N - 1]]))
        for r in rows.tolist():
            tgt, w, d = net.csr(r, 1)
            ot, ow, od = oracle.gen_rows(cfg, r, 1)
            assert np.array_equal(tgt, ot), r
            assert np.array_equal(w.view(np.uint32), ow.view(np.uint32)), r
            assert np.array_equal(d, od), r
        net.step(1)
        st, ids = net.read_spikes()
        s = net.state()
        spiked = set(ids.tolist())
        k = oracle.constants(cfg)
        sample = rng.integers(0, N, 3000)
        for i in sample.tolist():
            n_ext, forced = oracle.drive(cfg, i, 0)
            V, c, ref, sp = oracle.lif_update(cfg, oracle.initial_V(cfg, i), 0.0, 0,
                                              (i % M) < k["n_exc"], n_ext * k["J_ext_fx"], forced)
            assert np.float32(V) == s["V"][i] and np.float32(c) == s["c"][i] and ref == s["ref"][i], i
            assert sp == (i in spiked), i
        assert np.all(st == 0) and np.all(np.diff(ids.astype(np.int64)) > 0)
        # the ring after delivering every spike of step 0, recomputed from oracle rows
        expect = np.zeros((net.D, N), np.int64)
        scale = float(2 ** cfg["fx_shift"])
        for i in ids.tolist():
            ot, ow, od = oracle.gen_rows(cfg, i, 1)
            np.add.at(expect, (od.astype(np.int64) % net.D, ot.astype(np.int64)),
                      np.rint(ow.astype(np.float64) * scale).astype(np.int64))
        ring = s["ring"].astype(np.int64)
        expect[0] = 0  # slot 0 was consumed by step 0
        assert np.array_equal(ring, expect)
        # a longer run keeps the invariants
        net.clear_raster()
        net.set_schedule(schedule)
        net.step(200)
        st, ids = net.read_spikes()
        stats = net.stats()
        assert stats["rec_events"] == stats["n_spikes"] * K
        key = st.astype(np.int64) * N + ids
        assert np.all(np.diff(key) > 0)
        rate = len(st) / (N * 200) * 1000.0
        assert 0.5 * cfg["imposed_rate_hz"] < rate < 2.0 * cfg["imposed_rate_hz"] + 5.0


def test_full_size_gauss_24x24_k1125(snn):
    _full_size_check(snn, W.gauss_24x24_k1125(seed=1, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ), schedule=2)


def test_full_size_schedules_agree(snn):
    """The 24x24 Gaussian network run 60 steps with each schedule: identical state."""
    cfg = W.gauss_24x24_k1125(seed=3, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ, table_layout="grouped")
    out = []
    for schedule in (0, 2, 3, 4, 5):
        with snn.Network(cfg, raster_capacity=1 << 20) as net:
            net.set_schedule(schedule)
            net.step(60)
            st = net.state()
            out.append((net.read_spikes(), st["V"], st["ring"], net.stats()))
    (ra, Va, ga, sa) = out[0]
    for (rb, Vb, gb, sb) in out[1:]:
        assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
        assert np.array_equal(Va, Vb) and np.array_equal(ga, gb)
        assert all(sa[k] == sb[k] for k in ("n_spikes", "rec_events", "ext_events", "steps"))


def test_full_size_exp_24x24_k2250_bf16(snn):
    _full_size_check(snn, W.exp_24x24_k2250(seed=2, imposed_rate_hz=W.PAPER_RATE_EXP_HZ), n_rows=600)


def test_schedule_3_needs_the_grouped_layout(snn):
    with snn.Network(W.small()) as net:
        with pytest.raises(snn.SnnError, match="GROUPED"):
            net.set_schedule(3)


def test_kernel_timing_counts_sampled_launches(snn):
    cfg = W.small(grid=3, M=100, K=60, seed=8, imposed_rate_hz=30.0)
    with snn.Network(cfg) as net:
        net.set_timing(3)
        net.step(30)
        kt = net.kernel_time()
        assert kt["deliver_launches"] == 10 and kt["neuron_launches"] == 10
        assert kt["deliver_ms"] > 0 and kt["neuron_ms"] > 0
        net.set_timing(0)
        net.step(5)
        assert net.kernel_time()["deliver_launches"] == 10
        net.set_schedule(2)
        net.set_timing(1)
        net.step(20)
        net.step(7)
        kt = net.kernel_time()
        assert kt["persistent_launches"] == 2 and kt["persistent_ms"] > 0


def test_bounded_barrier_wait_reports_timeout(snn):
    """A grid-barrier arrival that never comes: every wait runs out after the
    limit, the launch returns, the host reads SNN_ETIMEOUT, the context stays usable."""
    cfg = W.small(grid=2, M=64, K=10, seed=1, imposed_rate_hz=50.0)
    with snn.Network(cfg) as net:
        net.set_schedule(2)
        net.set_wait_limit(2_000_000)  # 2 ms
        net.set_barrier_extra(1)
        net.step(5)
        with pytest.raises(snn.SnnError, match="SNN_ETIMEOUT"):
            net.stats()
        net.clear_error()
        net.set_barrier_extra(0)
    with snn.Network(cfg) as net2:
        net2.set_schedule(2)
        net2.step(10)
        ref = oracle.OracleNet(cfg)
        ref.step(10)
        _compare(net2, ref)


def test_autotune_leaves_the_simulation_unchanged(snn, tmp_path):
    cfg = dict(W.small(grid=3, M=200, K=150, seed=3, imposed_rate_hz=50.0), table_layout="grouped")
    cache = str(tmp_path / "tune.txt")
    with snn.Network(cfg) as net:
        net.step(20)
        sched, block, ms = net.autotune(trial_steps=15, cache_path=cache)
        assert sched in (0, 1, 2, 3, 4, 5) and ms > 0
        net.step(30)
        ref = oracle.OracleNet(cfg)
        ref.step(50)
        _compare(net, ref)
    with snn.Network(cfg) as net2:  # the cached choice is reused
        s2, b2, ms2 = net2.autotune(trial_steps=15, cache_path=cache)
        assert (s2, b2) == (sched, block) and ms2 == -1.0


def test_allocation_failure_is_reported_and_releases_everything(snn):
    import ctypes
    L = snn.load()
    live = {}
    calls = {"n": 0}
    import torch

    def alloc(size, ctx):
        calls["n"] += 1
        if calls["n"] == 6:  # fail the sixth allocation
            return None
        p = torch.cuda.caching_allocator_alloc(int(size))
        live[p] = size
        return p

    def free(ptr, ctx):
        live.pop(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = snn.ALLOC_FN(alloc), snn.FREE_FN(free)
    c = snn.config(W.small())
    h = ctypes.c_void_p()
    st = L.snn_build_network(ctypes.byref(c), fa, ff, None, None, ctypes.byref(h))
    assert st == snn.SNN_ENOMEM and h.value is None
    assert live == {}  # every block obtained before the failure was returned


def test_table_one_48x48_grid_runs_and_matches_sampled_rows(snn):
    """Table I's 48x48 grid (2.88 M neurons, 3.24 G synapses): sampled rows equal
    the oracle's, 50 persistent steps keep the invariants."""
    cfg = W.gauss_48x48_k1125(seed=4, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ)
    rng = np.random.default_rng(1)
    with snn.Network(cfg, raster_capacity=1 << 22) as net:
        assert net.N == 48 * 48 * 1250
        for r in rng.integers(0, net.N, 200).tolist() + [net.N - 1]:
            tgt, w, d = net.csr(r, 1)
            ot, ow, od = oracle.gen_rows(cfg, r, 1)
            assert np.array_equal(tgt, ot) and np.array_equal(w.view(np.uint32), ow.view(np.uint32))
            assert np.array_equal(d, od)
        net.set_schedule(2)
        net.step(50)
        st, ids = net.read_spikes()
        s = net.stats()
        assert s["rec_events"] == s["n_spikes"] * 1125 and len(st) == s["n_spikes"]
        assert np.all(np.diff(st.astype(np.int64) * net.N + ids) > 0)
        rate = s["n_spikes"] / (net.N * 50) * 1000.0
        assert 4.0 < rate < 12.0


def test_slow_wave_grid_tables(snn):
    cfg = dict(W.swa_48x48(), neurons_per_module=2, K=8)
    with snn.Network(cfg) as net:
        T, TM, cnt = net.cdf()
    for m in (0, 47, 48 * 24 + 24, 48 * 48 - 1):
        oT, oTM, _ = oracle.cdf_table(cfg, m)
        assert cnt[m] == len(oT) and np.array_equal(T[m, :len(oT)], oT) and np.array_equal(TM[m, :len(oT)], oTM)


BAND_CASES = {
    "gauss_grouped": lambda: W.small(grid=6, M=100, K=150, seed=31, imposed_rate_hz=30.0, table_layout="grouped"),
    "exp_grouped_bf16": lambda: dict(W.small(grid=5, M=60, K=200, lateral="exp", seed=32, weight_dtype="bf16",
                                             imposed_rate_hz=35.0, table_layout="grouped"), grid_h=7),
    "pairwise_gauss": lambda: W.pairwise(grid=8, M=60, seed=33, imposed_rate_hz=25.0),
    "pairwise_exp": lambda: W.pairwise(grid=9, M=30, lateral="exp", seed=34, imposed_rate_hz=35.0),
}


@pytest.mark.parametrize("resident", [True, False])
def test_resident_state_bit_exact(snn, resident):
    """Schedule 2 with the neuron state in shared memory through each launch,
    and with it in global memory: both give the oracle's results, across
    launch boundaries (the state is written back and read again) and with a
    snapshot taken between launches."""
    cfg = W.small(grid=4, M=250, K=120, seed=41, imposed_rate_hz=30.0, ext_rate_hz=3000.0)
    ref = oracle.OracleNet(cfg)
    ref.step(90)
    with snn.Network(cfg, raster_capacity=1 << 22) as net:
        assert net.set_resident_state(resident) == resident
        net.set_schedule(2)
        net.step(40)
        blob = net.snapshot()
        net.step(50)
        n = _compare(net, ref)
        with snn.Network(cfg, raster_capacity=1 << 22) as other:
            other.restore(blob)
            other.set_schedule(2)
            other.step(50)
            a, b = other.state(), net.state()
            for k in ("V", "c", "ref", "ring"):
                assert np.array_equal(a[k], b[k]), k
    assert n > 200


def test_resident_state_48x48_equals_per_step_kernels(snn):
    """Table I's 48x48 grid keeps 4,700 quads (171 KB) of state per CTA in
    shared memory: 30 persistent steps equal 30 steps of the per-step kernels
    (state in global memory), spike for spike."""
    cfg = W.gauss_48x48_k1125(seed=5, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ)
    out = []
    for schedule in (0, 2):
        with snn.Network(cfg, raster_capacity=1 << 22) as net:
            if schedule == 2:
                assert net.set_resident_state(True)
            net.set_schedule(schedule)
            net.step(30)
            s = net.state()
            out.append((net.read_spikes(), s["V"], s["c"], s["ref"]))
    (ra, Va, ca, fa), (rb, Vb, cb, fb) = out
    assert len(ra[0]) > 1000
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
    assert np.array_equal(Va.view(np.uint32), Vb.view(np.uint32)) and np.array_equal(ca, cb)
    assert np.array_equal(fa, fb)


@pytest.mark.parametrize("name", sorted(BAND_CASES))
def test_banded_delivery_bit_exact(snn, name):
    """Delivery in bands of target module rows (each band's ring columns
    L2-resident on large grids) gives the oracle's results for every band
    count."""
    cfg = BAND_CASES[name]()
    steps = 80
    ref = oracle.OracleNet(cfg)
    ref.step(steps)
    for bands in (1, 2, 3, cfg["grid_h"]):
        with snn.Network(cfg, raster_capacity=1 << 22) as net:
            assert net.set_bands(bands) == bands
            net.set_schedule(2)
            net.step(steps // 2)
            net.step(steps - steps // 2)
            n = _compare(net, ref)
    assert n > 200


def test_band_choice_and_errors(snn):
    with snn.Network(W.small(grid=3, M=50, K=20)) as net:  # draw layout: no segment index
        assert net.set_bands(0) == 1
        with pytest.raises(snn.SnnError, match="segment index"):
            net.set_bands(2)
    with snn.Network(W.small(grid=3, M=50, K=20, table_layout="grouped")) as net:
        assert net.set_bands(0) == 1  # a 13 KB ring fits in L2
        with pytest.raises(snn.SnnError, match="grid_h"):
            net.set_bands(4)
    # Table I's 48x48 grid: a 242 MB ring is delivered in ceil(ring / (L2 / 2)) bands by default
    import torch
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    with snn.Network(W.gauss_48x48_k1125(seed=2, table_layout="grouped", imposed_rate_hz=7.5)) as net:
        ring = 21 * ((net.N + 1023) // 1024 * 1024) * 4
        assert net.set_bands(0) == min(-(-ring // (l2 // 2)), 48 // 7)


def _random_configs(n=8, seed=2026):
    """Seeded random descriptions spanning both laws, both kernels, both weight
    types, odd grid shapes, module sizes that are not multiples of the block,
    uniform and Gaussian efficacies, uniform and exponential delays, rates."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        lateral = "gauss" if rng.random() < 0.5 else "exp"
        gw, gh = int(rng.integers(1, 7)), int(rng.integers(1, 7))
        M = int(rng.integers(7, 160))
        extra = {"grid_h": gh, "weight_dtype": "bf16" if rng.random() < 0.4 else "f32",
                 "imposed_rate_hz": float(rng.choice([0.0, 7.5, 35.0, 80.0])),
                 "ext_rate_hz": float(rng.choice([0.0, 1500.0, 4000.0])),
                 "weight_dist": "gauss" if rng.random() < 0.5 else "uniform",
                 "delay_dist": "exp" if rng.random() < 0.5 else "uniform",
                 "d_exc_hi": int(rng.integers(1, 25)), "seed": int(rng.integers(1, 1 << 40)),
                 "delay_tau_ms": float(rng.uniform(1.0, 10.0)), "w_exc_sd": float(rng.uniform(0.0, 0.1)),
                 "w_inh_sd": float(rng.uniform(0.0, 0.4))}
        if rng.random() < 0.5:
            cfg = W.pairwise(grid=gw, M=M, lateral=lateral, **extra)
        else:
            cfg = W.small(grid=gw, M=M, K=int(rng.integers(0, 300)), lateral=lateral, **extra)
            cfg["table_layout"] = "grouped" if rng.random() < 0.5 else "draw"
        out.append(cfg)
    return out


@pytest.mark.parametrize("k", range(8))
def test_random_descriptions_bit_exact(snn, k):
    """Seeded random descriptions: every schedule that supports the description
    equals the oracle after 120 steps."""
    cfg = _random_configs()[k]
    ref = oracle.OracleNet(cfg)
    ref.step(120)
    schedules = [0, 1, 2, 4] + ([3] if cfg.get("table_layout") == "grouped" else [])
    for schedule in schedules:
        with snn.Network(cfg, raster_capacity=1 << 22) as net:
            try:
                net.set_schedule(schedule)
            except snn.SnnError:
                assert schedule == 3  # the tile may not fit in shared memory
                continue
            net.step(47)
            net.step(73)
            _compare(net, ref)
