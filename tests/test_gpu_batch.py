"""Batched execution: independent networks advanced in one persistent launch
must each equal the network run alone (here: the oracle), bit for bit."""
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


def _cases():
    return [
        W.small(grid=2, M=120, K=77, seed=5, imposed_rate_hz=30.0, ext_rate_hz=3000.0),
        W.small(grid=3, M=100, K=200, lateral="exp", seed=6, weight_dtype="bf16", imposed_rate_hz=35.0),
        W.small(grid=4, M=50, K=150, seed=7, ext_rate_hz=5000.0),
        dict(W.small(grid=3, M=333, K=37, seed=9, imposed_rate_hz=40.0), grid_h=2),
        W.small(grid=2, M=64, K=10, seed=1, ext_rate_hz=0.0),
        W.gauss_4x4_k1000(seed=2, imposed_rate_hz=7.5),
    ]


def _check(net, ref):
    st, ids = net.read_spikes()
    rs, ri = ref.raster()
    assert np.array_equal(st, rs) and np.array_equal(ids, ri)
    a, b = net.state(), ref.state()
    for k in ("V", "c", "ref", "ring"):
        assert np.array_equal(a[k], b[k]), k
    assert a["t"] == ref.t
    s = net.stats()
    assert s["n_spikes"] == ref.stats()["spikes"] and s["ext_events"] == ref.stats()["ext_events"]


@pytest.mark.parametrize("mode", ["groups", "global"])
@pytest.mark.parametrize("graph,waves", [(False, 1), (True, 1), (True, 3)])
def test_batch_equals_each_network_alone(snn, graph, waves, mode):
    cfgs = _cases()
    nets = [snn.Network(c, raster_capacity=1 << 20) for c in cfgs]
    refs = [oracle.OracleNet(c) for c in cfgs]
    with snn.Batch(nets) as batch:
        batch.set_mode(mode)
        batch.set_graph(graph)
        if waves > 1:  # a ring budget that gives every network its own launch
            batch.set_ring_budget(1)
            assert batch.waves()[0] == len(nets)
        plans = [[60, 45, 60, 0, 30, 50], [10, 10, 0, 25, 10, 10], [10, 10, 0, 25, 10, 10]]
        for steps in plans:
            batch.step(steps)
            for r, n in zip(refs, steps):
                r.step(n)
        for net, ref in zip(nets, refs):
            _check(net, ref)
        ms, launches = batch.time()
        assert launches == len(plans) and ms > 0
    for n in nets:
        n.close()


def test_batch_of_one_equals_the_persistent_schedule(snn):
    cfg = W.small(grid=3, M=100, K=60, seed=8, imposed_rate_hz=30.0)
    with snn.Network(cfg) as a, snn.Network(cfg) as b:
        a.set_schedule(2)
        a.step(70)
        with snn.Batch([b]) as batch:
            batch.step([70])
        sa, sb = a.state(), b.state()
        for k in ("V", "c", "ref", "ring", "t"):
            assert np.array_equal(sa[k], sb[k]), k
        assert all(np.array_equal(x, y) for x, y in zip(a.read_spikes(), b.read_spikes()))


def test_batch_barrier_wait_runs_out(snn):
    """Global wave: one pair of barriers for the wave, so a barrier that cannot
    be passed (a test knob expecting one arrival too many) stops every
    network of the wave."""
    cfgs = _cases()[:2]
    nets = [snn.Network(c) for c in cfgs]
    nets[0].set_wait_limit(2_000_000)
    nets[1].set_barrier_extra(1)
    with snn.Batch(nets) as batch:
        batch.set_mode("global")
        batch.step([5, 5])
    for n in nets:
        with pytest.raises(snn.SnnError, match="SNN_ETIMEOUT"):
            n.stats()
        n.close()


def test_grouped_barrier_wait_runs_out_in_its_group_only(snn):
    """Grouped wave: each network passes its own barriers, so only the network
    whose barrier cannot be passed reports the timeout; the others run on and
    still equal the oracle."""
    cfgs = _cases()[:3]
    nets = [snn.Network(c, raster_capacity=1 << 20) for c in cfgs]
    refs = [oracle.OracleNet(c) for c in cfgs]
    for n in nets:
        n.set_wait_limit(2_000_000)
    nets[1].set_barrier_extra(1)
    with snn.Batch(nets) as batch:
        batch.step([30, 30, 30])
        assert all(g > 0 for g in batch.groups())
    with pytest.raises(snn.SnnError, match="SNN_ETIMEOUT"):
        nets[1].stats()
    for i in (0, 2):
        refs[i].step(30)
        _check(nets[i], refs[i])
    for n in nets:
        n.close()


def test_groups_cover_the_active_networks(snn):
    """Every network that runs gets a group, idle ones none, and the groups
    of a wave never take more CTAs than the grid (one per SM); the split
    follows the work (a network 16x larger gets more CTAs)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cfgs = [W.small(grid=8, M=1250, K=1125, seed=s, imposed_rate_hz=20.0) for s in range(3)]
    cfgs.append(W.small(grid=2, M=1250, K=1125, seed=9, imposed_rate_hz=20.0))
    nets = [snn.Network(c) for c in cfgs]
    with snn.Batch(nets) as batch:
        batch.set_graph(True)
        for steps in ([20, 20, 0, 20], [40, 40, 40, 40], [40, 40, 40, 40]):
            batch.step(steps)
            g = batch.groups()
            assert all((x > 0) == (s > 0) for x, s in zip(g, steps)) and sum(g) <= sms
        assert g[3] < min(g[:3])
        batch.set_mode("global")
        batch.step([5, 5, 5, 5])
        assert batch.groups() == [0, 0, 0, 0]
    for n in nets:
        n.close()


def test_batch_rejects_repeated_networks(snn):
    net = snn.Network(W.small())
    with pytest.raises(snn.SnnError, match="twice"):
        snn.Batch([net, net])
    net.close()


def test_waves_that_cannot_be_grouped_run_global(snn):
    """A wave holding a banded network, and a wave with more networks than
    SMs, run in the global layout even in groups mode: every network still
    equals the oracle, and none of them reports a group."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    banded = W.small(grid=4, M=60, K=80, seed=51, imposed_rate_hz=30.0, table_layout="grouped")
    cfgs = [banded, W.small(grid=2, M=50, K=40, seed=52, imposed_rate_hz=30.0)]
    nets = [snn.Network(c, raster_capacity=1 << 20) for c in cfgs]
    assert nets[0].set_bands(2) == 2
    refs = [oracle.OracleNet(c) for c in cfgs]
    with snn.Batch(nets) as batch:
        batch.step([40, 40])
        assert batch.groups() == [0, 0]
    for net, ref in zip(nets, refs):
        ref.step(40)
        _check(net, ref)
        net.close()
    # more networks than SMs in one wave
    many = [W.small(grid=1, M=12, K=6, seed=100 + i, imposed_rate_hz=60.0) for i in range(sms + 3)]
    nets = [snn.Network(c, raster_capacity=1 << 12) for c in many]
    with snn.Batch(nets) as batch:
        assert batch.waves()[0] == 1
        batch.step([25] * len(nets))
        assert set(batch.groups()) == {0}
    for i in (0, len(nets) // 2, len(nets) - 1):
        ref = oracle.OracleNet(many[i])
        ref.step(25)
        _check(nets[i], ref)
    for n in nets:
        n.close()


def test_grouped_batch_of_both_laws_and_weight_types(snn):
    """A grouped wave mixing the per-pair law (bf16 and f32), the fixed law and
    a network with an imposed rate of 0 (driven only by its Poisson input),
    over several calls with changing step counts (the split is re-planned from
    the measured group times each call): bit-exact against the oracle."""
    cfgs = [W.pairwise(grid=5, M=80, seed=61, imposed_rate_hz=20.0, weight_dtype="bf16"),
            W.pairwise(grid=4, M=90, lateral="exp", seed=62, imposed_rate_hz=35.0),
            W.small(grid=5, M=100, K=150, seed=63, imposed_rate_hz=7.5, weight_dtype="bf16"),
            W.small(grid=3, M=120, K=90, seed=64, ext_rate_hz=4000.0)]
    nets = [snn.Network(c, raster_capacity=1 << 20) for c in cfgs]
    refs = [oracle.OracleNet(c) for c in cfgs]
    with snn.Batch(nets) as batch:
        batch.set_graph(True)
        for steps in ([30, 30, 30, 30], [50, 10, 0, 35], [64, 64, 64, 64]):
            batch.step(steps)
            assert all((g > 0) == (s > 0) for g, s in zip(batch.groups(), steps))
            for r, k in zip(refs, steps):
                r.step(k)
    for net, ref in zip(nets, refs):
        _check(net, ref)
        net.close()


@pytest.mark.parametrize("shape", [0, 1])
def test_global_layout_launch_shapes_equal_the_oracle(snn, shape):
    """Both launch shapes of the global layout (2 CTAs per SM x 4 tasks in
    flight, 1 CTA per SM x 6) give the oracle's results."""
    cfgs = _cases()
    nets = [snn.Network(c, raster_capacity=1 << 20) for c in cfgs]
    refs = [oracle.OracleNet(c) for c in cfgs]
    with snn.Batch(nets) as batch:
        batch.set_mode("global")
        batch.set_shape(shape)
        batch.set_graph(True)
        for steps in ([40, 40, 40, 40, 40, 40], [7, 0, 19, 3, 11, 5]):
            batch.step(steps)
            for r, n in zip(refs, steps):
                r.step(n)
    for net, ref in zip(nets, refs):
        _check(net, ref)
        net.close()


def test_autotuned_batch_changes_no_result(snn, tmp_path):
    """The tuner runs every candidate layout, shape and ring budget from one
    snapshot and restores it: afterwards the batch continues exactly as the
    oracle does; a second call finds the choice in the cache."""
    cfgs = _cases()
    nets = [snn.Network(c, raster_capacity=1 << 20) for c in cfgs]
    refs = [oracle.OracleNet(c) for c in cfgs]
    cache = str(tmp_path / "tune.txt")
    with snn.Batch(nets) as batch:
        batch.step([15] * len(nets))
        for r in refs:
            r.step(15)
        got = batch.autotune(trial_steps=20, cache_path=cache)
        assert got["mode"] in ("groups", "global") and got["shape"] in (0, 1) and got["ms_per_step"] > 0
        again = batch.autotune(trial_steps=20, cache_path=cache)
        assert again["ms_per_step"] == -1.0 and (again["mode"], again["shape"], again["ring_budget"]) == \
            (got["mode"], got["shape"], got["ring_budget"])
        batch.set_graph(True)
        batch.step([30, 10, 30, 0, 30, 25])
        for r, n in zip(refs, [30, 10, 30, 0, 30, 25]):
            r.step(n)
    for net, ref in zip(nets, refs):
        _check(net, ref)
        net.close()
