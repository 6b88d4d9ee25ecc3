"""Pin the oracle's external Poisson drive (Sec. III-A) and its spike delivery
(flow steps 2-4 of Sec. II-A, integer delays of Sec. II-B)."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1803_08833_gb300 import workloads as W


def test_poisson_table_is_the_poisson_cdf():
    cfg = W.small()
    k = oracle.constants(cfg)
    lam = cfg["ext_rate_hz"] * cfg["dt_ms"] / 1000.0
    assert lam == 1.5
    cdf = stats.poisson.cdf(np.arange(len(k["pois"])), lam)
    ref = np.floor(cdf * 2.0 ** 32)
    assert np.all(np.abs(np.array(k["pois"], dtype=np.float64) - ref) <= 1.0)
    # counts run up to len(table); the mass above that is below one part in 2^32
    L = len(k["pois"])
    assert stats.poisson.sf(L, lam) < 2.0 ** -32 < stats.poisson.sf(L - 1, lam)


def test_poisson_count_boundaries():
    cfg = W.small()
    P = oracle.constants(cfg)["pois"]
    assert oracle.poisson_count(cfg, 0) == 0
    assert oracle.poisson_count(cfg, P[0] - 1) == 0
    assert oracle.poisson_count(cfg, P[0]) == 1
    assert oracle.poisson_count(cfg, P[3]) == 4
    assert oracle.poisson_count(cfg, 2 ** 32 - 1) == len(P)
    cfg0 = W.small(ext_rate_hz=0.0)
    assert oracle.constants(cfg0)["pois"] == []
    assert oracle.poisson_count(cfg0, 2 ** 32 - 1) == 0


def test_drive_mean_variance_and_pmf():
    """Counts drawn from Philox(seed; i, t, DRIVE) are Poisson(nu_ext dt)."""
    cfg = W.small()
    key = [cfg["seed"] & 0xFFFFFFFF, cfg["seed"] >> 32]
    n = []
    for i in range(200):
        for t in range(150):
            u0 = oracle.philox([i, t, 1, 0], key)[0]
            n.append(oracle.poisson_count(cfg, u0))
    n = np.array(n)
    lam = 1.5
    se = math.sqrt(lam / n.size)
    assert abs(n.mean() - lam) < 4 * se
    assert abs(n.var() - lam) < 4 * math.sqrt(2 * lam ** 2 / n.size + lam / n.size)
    obs = np.bincount(n, minlength=8)[:7]
    exp = stats.poisson.pmf(np.arange(7), lam) * n.size
    obs = np.append(obs, n.size - obs.sum())
    exp = np.append(exp, n.size - exp.sum())
    assert stats.chisquare(obs, exp).pvalue > 1e-3


def test_network_external_event_count():
    cfg = W.small(grid=2, M=100, K=10)
    net = oracle.OracleNet(cfg)
    net.step(400)
    ext = net.stats()["ext_events"]
    n = net.N * 400
    assert abs(ext / n - 1.5) < 4 * math.sqrt(1.5 / n)


def _quiet(cfg):
    """No drive, E = 0, no adaptation: membrane moves only through recurrent input."""
    cfg = dict(cfg, ext_rate_hz=0.0, imposed_rate_hz=0.0, alpha_c=0.0, E_mV=0.0)
    return cfg


def test_arrival_step_and_amplitude_of_one_spike():
    """One neuron spikes at step 0; each target first moves at step d (its
    synapse's delay) by exactly the fixed-point sum of the weights arriving then."""
    for src in (3, 37):  # one excitatory (delays 1..20), one inhibitory (delay 1)
        cfg = _quiet(W.small(grid=2, M=40, K=60, seed=9))
        net = oracle.OracleNet(cfg)
        N = net.N
        V = np.zeros(N, np.float32)
        V[src] = 100.0
        net.set_state(V=V, c=np.zeros(N, np.float32), ref=np.zeros(N, np.uint8))
        tgt, w, d = net.csr()
        K = net.K
        row = slice(src * K, (src + 1) * K)
        tg, ww, dd = tgt[row], w[row], d[row]
        trace = []
        for t in range(22):
            net.step(1)
            trace.append(net.state()["V"].copy())
        st, ids = net.raster()
        assert st.tolist() == [0] and ids.tolist() == [src]
        trace = np.array(trace)
        for j in set(tg.tolist()) - {src}:
            dmin = dd[tg == j].min()
            moved = np.nonzero(trace[:, j] != 0.0)[0]
            assert moved[0] == dmin, (j, moved[0], dmin)
            fx = np.rint(ww[(tg == j) & (dd == dmin)].astype(np.float64) * 65536.0).sum()
            assert trace[dmin, j] == np.float32(fx / 65536.0)
        untouched = np.setdiff1d(np.arange(N), np.append(tg, src))
        assert np.all(trace[:, untouched] == 0.0)


def test_ring_holds_fixed_point_sums_at_t_plus_d():
    cfg = _quiet(W.small(grid=2, M=40, K=60, seed=4))
    net = oracle.OracleNet(cfg)
    N, K, D = net.N, net.K, net.D
    V = np.zeros(N, np.float32)
    srcs = [1, 2, 50, 77, 120]
    V[srcs] = 100.0
    net.set_state(V=V, c=np.zeros(N, np.float32), ref=np.zeros(N, np.uint8))
    net.step(1)
    ring = net.state()["ring"]
    tgt, w, d = net.csr()
    expect = np.zeros((D, N), np.int64)
    for s in srcs:
        for k in range(K):
            e = s * K + k
            expect[(0 + d[e]) % D, tgt[e]] += int(np.rint(np.float64(w[e]) * 65536.0))
    assert np.array_equal(ring.astype(np.int64), expect)


def test_delivery_order_does_not_change_anything():
    cfg = W.small(grid=3, M=60, K=80, seed=21, imposed_rate_hz=40.0)
    a = oracle.OracleNet(cfg)
    b = oracle.OracleNet(cfg)
    b.set_delivery_shuffle(12345)
    a.step(60)
    b.step(60)
    sa, sb = a.state(), b.state()
    for k in ("V", "c", "ref", "ring"):
        assert np.array_equal(sa[k], sb[k]), k
    assert all(np.array_equal(x, y) for x, y in zip(a.raster(), b.raster()))
    assert a.stats()["spikes"] > 100


def test_imposed_rate_and_counters():
    rate = 35.0
    cfg = W.small(grid=2, M=250, K=20, seed=8, imposed_rate_hz=rate, ext_rate_hz=0.0)
    net = oracle.OracleNet(cfg)
    T = 400
    net.step(T)
    s = net.stats()
    p = rate / 1000.0
    # a neuron is forced with probability p unless refractory (2 steps after a spike)
    expect = net.N * T * p / (1 + 2 * p)
    assert abs(s["spikes"] - expect) < 5 * math.sqrt(expect)
    assert s["rec_events"] == s["spikes"] * net.K
    st, ids = net.raster()
    assert len(st) == s["spikes"]
    key = st.astype(np.int64) * net.N + ids
    assert np.all(np.diff(key) > 0)  # sorted by (step, id), no duplicates


def test_fp64_mode_follows_fp32_mode():
    cfg = W.small(grid=3, M=100, K=50, seed=6, ext_rate_hz=4000.0)
    a = oracle.OracleNet(cfg)
    b = oracle.OracleNet(cfg, fp64=True)
    a.step(300)
    b.step(300)
    ra, rb = a.stats()["spikes"], b.stats()["spikes"]
    assert ra > 200
    assert abs(ra - rb) < 0.05 * ra
    assert a.stats()["ext_events"] == b.stats()["ext_events"]
