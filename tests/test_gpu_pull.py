"""Schedule 5 (band-owned delay windows filled by pulling row ranges) against
the oracle.

Every CTA owns a band of neurons, keeps the input of its next W steps in
shared memory and reads, from each spiking row whose source module's stencil
reaches the band, the contiguous range of synapses that targets the band's
modules (the grouped layout orders each row by target module).  Near events
go into the window, far ones into the ring; one grid barrier per step.  None
of that may change a result: spike raster, V, c, refractory counters, the
whole ring and the counters must equal the oracle bit for bit, for any
window, both lateral kernels, both connection laws, ragged bands and modules,
and across launches, snapshots and schedule switches.
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


def _grouped(cfg):
    return dict(cfg, table_layout="grouped")


CASES = {
    # bands of a few modules; the 3-sigma stencil reaches every module of the grid
    "gauss_imposed": (lambda: _grouped(W.small(grid=4, M=250, K=300, seed=3, imposed_rate_hz=40.0)), 150),
    # long-range kernel, bf16 weights, more modules than bands cover with one run each
    "exp_bf16": (lambda: _grouped(W.small(grid=6, M=120, K=400, lateral="exp", seed=5, weight_dtype="bf16",
                                          imposed_rate_hz=35.0)), 120),
    # M not a multiple of 4 (modules split inside quads), K not a multiple of 8, short delays
    "ragged_delays": (lambda: _grouped(dict(W.small(grid=3, M=333, K=37, seed=9, imposed_rate_hz=40.0, d_exc_hi=7),
                                            grid_h=2)), 150),
    # a short cutoff: stencils reach only some of the modules, many bands have few runs
    "short_cutoff": (lambda: _grouped(dict(W.small(grid=7, M=77, K=60, seed=12, imposed_rate_hz=45.0),
                                           grid_h=9, cutoff_um=120.0)), 120),
    # external drive only, at the specified 4x4 network's size
    "drive": (lambda: _grouped(W.gauss_4x4_k1000(seed=2, ext_rate_hz=5000.0)), 200),
    # the per-pair law (rows of variable length, grouped by stencil offset by construction)
    "pairwise_gauss": (lambda: W.pairwise(grid=4, M=150, seed=6, imposed_rate_hz=30.0), 100),
    "pairwise_exp_bf16": (lambda: dict(W.pairwise(grid=5, M=90, lateral="exp", seed=8, weight_dtype="bf16",
                                                  imposed_rate_hz=35.0), grid_h=3), 100),
}


@pytest.mark.parametrize("band_mode", [1, 2])
@pytest.mark.parametrize("window", [0, 1, 2, 5])
@pytest.mark.parametrize("name", sorted(CASES))
def test_windows_equal_oracle(snn, name, window, band_mode):
    """Window 1 sends every event of delay > 1 to the ring; the default keeps
    most of them in shared memory.  Band mode 1 splits modules between bands
    (M = 250, 333, 77 leave modules inside quads), mode 2 cuts only at module
    boundaries on a multiple of 4 neurons (every module for M = 1000, every
    second for M = 250 and 120, every fourth for M = 333 and 77)."""
    make, steps = CASES[name]
    cfg = make()
    ref = oracle.OracleNet(cfg)
    ref.step(steps)
    with snn.Network(cfg, raster_capacity=1 << 22) as net:
        net.set_schedule(5)
        wmax = net.set_pull_window(0, band_mode)
        assert net.pull_band_mode == band_mode
        if window > wmax:
            pytest.skip("window %d does not fit (max %d)" % (window, wmax))
        assert net.set_pull_window(window, band_mode) == (window or wmax)
        net.step(steps // 3)
        net.step(1)
        net.step(steps - steps // 3 - 1)
        n = _compare(net, ref)
    assert n > 500


def test_switching_schedules_and_snapshot(snn):
    """Pieces of schedule 5 between pieces of schedules 2, 4 and 0, and a
    snapshot taken after a schedule-5 launch, resume bit-exactly."""
    cfg = _grouped(W.small(grid=4, M=200, K=250, seed=11, imposed_rate_hz=25.0, ext_rate_hz=3000.0))
    ref = oracle.OracleNet(cfg)
    ref.step(140)
    with snn.Network(cfg, raster_capacity=1 << 22) as net:
        for sched, n in ((5, 17), (2, 23), (5, 1), (0, 9), (4, 5), (5, 25)):
            net.set_schedule(sched)
            net.step(n)
        blob = net.snapshot()
        with snn.Network(cfg, raster_capacity=1 << 22) as other:
            other.restore(blob)
            other.set_schedule(5)
            other.step(60)
            net.set_schedule(5)
            net.step(60)
            sa, sb = net.state(), other.state()
            for k in ("V", "c", "ref", "ring"):
                assert np.array_equal(sa[k], sb[k])
        _compare(net, ref)


@pytest.mark.parametrize("make,band_mode", [
    (lambda: W.gauss_24x24_k1125(seed=5, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ, table_layout="grouped"), 0),
    (lambda: W.gauss_24x24_k1125(seed=5, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ, table_layout="grouped"), 1),
    (lambda: W.exp_24x24_k2250(seed=4, imposed_rate_hz=W.PAPER_RATE_EXP_HZ, table_layout="grouped"), 0),
    (lambda: W.pairwise(grid=24, seed=3, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ), 0),
], ids=["gauss_24x24_k1125", "gauss_24x24_k1125_uniform_bands", "exp_24x24_k2250_bf16", "pairwise_24x24_gauss"])
def test_full_size_schedule_5_equals_schedule_2(snn, make, band_mode):
    """The 24x24 benchmark networks (720,000 neurons, 810 M and 1.6 G synapses)
    at the paper's rates, 200 steps in two calls: schedule 5 with its default
    window equals schedule 2 in raster, state, ring and counters.  The
    automatic bands of these networks are module-aligned (2 or 4 modules of
    1,250 neurons against 4,740 neurons per uniform band)."""
    cfg = make()
    out = []
    for sched in (2, 5):
        with snn.Network(cfg, raster_capacity=1 << 24) as net:
            net.set_schedule(sched)
            if sched == 5:
                assert net.set_pull_window(0, band_mode) >= 6  # most delays stay in shared memory on a GB300
                assert net.pull_band_mode == (band_mode or 2)
            net.step(120)
            net.step(80)
            st = net.state()
            out.append((net.read_spikes(), st["V"], st["c"], st["ref"], st["ring"], net.stats()))
    a, b = out
    assert np.array_equal(a[0][0], b[0][0]) and np.array_equal(a[0][1], b[0][1])
    for k in range(1, 5):
        assert np.array_equal(a[k], b[k])
    assert all(a[5][k] == b[5][k] for k in ("n_spikes", "rec_events", "ext_events", "steps"))
    assert a[5]["n_spikes"] > 500_000


def test_schedule_5_bounded_barrier_wait_reports_timeout(snn):
    cfg = _grouped(W.small(grid=2, M=64, K=10, seed=1, imposed_rate_hz=50.0))
    with snn.Network(cfg) as net:
        net.set_schedule(5)
        net.set_wait_limit(2_000_000)  # 2 ms
        net.set_barrier_extra(1)
        net.step(5)
        with pytest.raises(snn.SnnError, match="SNN_ETIMEOUT"):
            net.stats()
        net.clear_error()
        net.set_barrier_extra(0)
    with snn.Network(cfg) as net2:
        net2.set_schedule(5)
        net2.step(10)
        ref = oracle.OracleNet(cfg)
        ref.step(10)
        _compare(net2, ref)


def test_schedule_5_refuses_bands_beyond_tensor_memory(snn):
    """The band's neuron state stays in tensor memory (512 columns per SM: at
    most 7,168 quads a band on 16 warps).  100 x 100 modules of 440 neurons
    give bands of 29,040 (aligned) or 28,948 (uniform) neurons: a window row
    still fits in shared memory, the state does not, and the schedule is
    refused with the network left usable."""
    cfg = _grouped(W.small(grid=100, M=440, K=10, seed=4, imposed_rate_hz=20.0))
    with snn.Network(cfg) as net:
        with pytest.raises(snn.SnnError, match="tensor memory"):
            net.set_schedule(5)
        net.set_schedule(2)
        net.step(3)
        assert net.stats()["steps"] == 3


def test_schedule_5_argument_errors(snn):
    with snn.Network(W.small(grid=2, M=64, K=10, seed=1)) as net:  # draw-order rows
        with pytest.raises(snn.SnnError, match="GROUPED"):
            net.set_schedule(5)
    with snn.Network(_grouped(W.small(grid=2, M=64, K=10, seed=1))) as net:
        net.set_schedule(5)
        wmax = net.set_pull_window(0)
        with pytest.raises(snn.SnnError, match="window"):
            net.set_pull_window(wmax + 1)
        with pytest.raises(snn.SnnError, match="band_mode"):
            net.set_pull_window(0, 3)
