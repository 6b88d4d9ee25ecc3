"""Spike-timing dependent plasticity on the GPU against the oracle (Sec. II-A:
contributions at post-synaptic spikes and pre-synaptic arrivals, applied to
every synapse each period).  Everything is integer or the same IEEE float
expression on both sides, so the plastic weights, the accumulated changes,
the traces and the whole simulated state must be bit-exact, period after
period (the weights of one period feed the deliveries of the next)."""
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


CASES = {
    "gauss": (lambda: W.plastic(W.small(grid=3, M=120, K=80, seed=31, imposed_rate_hz=30.0, ext_rate_hz=3000.0),
                                stdp_period_steps=100, stdp_A_plus=0.02, stdp_A_minus=0.021), 250),
    "exp_grouped": (lambda: W.plastic(dict(W.small(grid=4, M=60, K=150, lateral="exp", seed=32, imposed_rate_hz=40.0),
                                           table_layout="grouped"), stdp_period_steps=70), 160),
    "pairwise": (lambda: W.plastic(W.pairwise(grid=3, M=50, seed=33, imposed_rate_hz=25.0),
                                   stdp_period_steps=60, stdp_w_max=0.35), 150),
    "ragged_short_delays": (lambda: W.plastic(dict(W.small(grid=3, M=77, K=37, seed=34, imposed_rate_hz=50.0,
                                                           d_exc_hi=4), grid_h=2),
                                              stdp_period_steps=50, stdp_tau_plus_ms=10.0, stdp_tau_minus_ms=30.0),
                            140),
}


def _grouped_order(cfg, tgt, K):
    """Permutation of draw-order rows into the grouped layout: each row stably
    sorted by the stencil position of its targets' modules (the order of the
    source module's target-module table)."""
    M = cfg["neurons_per_module"]
    N = len(tgt) // K
    perm = np.empty(len(tgt), np.int64)
    pos = {}
    for i in range(N):
        s = i // M
        if s not in pos:
            TM = oracle.cdf_table(cfg, s)[1]
            pos[s] = {int(m): j for j, m in enumerate(TM.tolist())}
        key = np.array([pos[s][int(t) // M] for t in tgt[i * K:(i + 1) * K]])
        perm[i * K:(i + 1) * K] = i * K + np.argsort(key, kind="stable")
    return perm


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("name", sorted(CASES))
def test_stdp_bit_exact_against_oracle(snn, name, schedule):
    make, steps = CASES[name]
    cfg = make()
    ref = oracle.OracleNet(cfg)
    w0 = ref.csr()[1].copy()
    ref.step(steps)
    with snn.Network(cfg, raster_capacity=1 << 22) as net:
        net.set_schedule(schedule)
        net.step(steps // 3)
        net.step(steps - steps // 3)
        st, ids = net.read_spikes()
        rs, ri = ref.raster()
        assert np.array_equal(st, rs) and np.array_equal(ids, ri), (len(st), len(rs))
        s, o = net.state(), ref.state()
        for k in ("V", "c", "ref", "ring"):
            assert np.array_equal(np.asarray(s[k]).view(np.uint8), np.asarray(o[k]).view(np.uint8)), k
        tgt, w, d = net.csr()
        otgt, ow, od = ref.csr()
        odelta, oy, ox = ref.stdp()
        changed = np.count_nonzero(ow != w0)  # draw order on both sides
        if cfg.get("table_layout") == "grouped":  # the GPU rows are stably grouped by target module
            perm = _grouped_order(cfg, otgt, net.K)
            otgt, ow, od, odelta = otgt[perm], ow[perm], od[perm], odelta[perm]
        assert np.array_equal(tgt, otgt) and np.array_equal(d, od)
        assert np.array_equal(w.view(np.uint32), ow.view(np.uint32))  # the plastic weights
        delta, y, x = net.stdp()
        assert np.array_equal(delta.astype(np.int64), odelta)
        assert np.array_equal(y.view(np.uint32), oy.view(np.uint32))
        assert np.array_equal(x.view(np.uint32), ox.view(np.uint32))
        a, b = net.stats(), ref.stats()
        assert a["n_spikes"] == b["spikes"] and a["rec_events"] == b["rec_events"]
    assert len(st) > 300
    assert changed > 100  # the periods changed weights
    assert np.count_nonzero(odelta) > 100    # and the open period has accumulated changes


def test_stdp_restrictions(snn):
    cfg = CASES["gauss"][0]()
    with snn.Network(cfg) as net:
        with pytest.raises(snn.SnnError, match="per-step schedules"):
            net.set_schedule(2)
        with pytest.raises(snn.SnnError, match="snapshots"):
            net.snapshot()
        with pytest.raises(snn.SnnError, match="batches"):
            snn.Batch([net])
    with pytest.raises(snn.SnnError, match="f32 weights"):
        snn.Network(dict(cfg, weight_dtype="bf16"))
    with snn.Network(W.small()) as plain:
        with pytest.raises(snn.SnnError, match="no plasticity"):
            plain.stdp()
