"""Pin the oracle's spike-timing dependent plasticity (Sec. II-A: STDP
contributions at every post-synaptic spike and every pre-synaptic arrival,
integrated into a long-term change of each synapse every period; the paper
gives no rule, this build's reading is pair-based with exponential traces).

The pin is the closed form of the rule over the whole raster: for a synapse
i -> j with delay d, its arrivals are a = t_i + d, and after T steps its change
is  A+ sum_{b, a < b} exp(-(b - a)/tau+) - A- sum_{a, b <= a} exp(-(a - b)/tau-)
over the post-synaptic spikes b of j -- computed here pair by pair from the
raster, independently of the oracle's traces and arrival queues."""
import math

import numpy as np

import oracle
from paper_1803_08833_gb300 import workloads as W


def _cfg(**kw):
    base = W.small(grid=2, M=40, K=25, seed=13, imposed_rate_hz=45.0, ext_rate_hz=2000.0)
    return W.plastic(base, **kw)


def _pair_sums(cfg, net, T):
    """Closed-form change (mV) of every synapse after steps 0 .. T-1."""
    tgt, w, d = net.csr()
    rp = net.row_ptr()
    st, ids = net.raster()
    spikes = [st[ids == i].astype(np.float64) for i in range(net.N)]
    Ap, Am = float(np.float32(cfg["stdp_A_plus"])), float(np.float32(cfg["stdp_A_minus"]))
    tp, tm = cfg["stdp_tau_plus_ms"], cfg["stdp_tau_minus_ms"]
    out = np.zeros(len(tgt))
    events = np.zeros(len(tgt), np.int64)
    M, n_exc = cfg["neurons_per_module"], oracle.constants(cfg)["n_exc"]
    for i in range(net.N):
        if i % M >= n_exc:
            continue  # inhibitory synapses are not plastic
        for e in range(int(rp[i]), int(rp[i + 1])):
            a = spikes[i] + d[e]
            a = a[a <= T - 1]  # arrivals processed within the run
            b = spikes[tgt[e]]
            if len(a) == 0 and len(b) == 0:
                continue
            diff = b[None, :] - a[:, None]  # b - a
            ltp = Ap * np.exp(-np.where(diff > 0, diff, np.inf) / tp).sum()
            ltd = Am * np.exp(-np.where(diff <= 0, -diff, np.inf) / tm).sum()
            out[e] = ltp - ltd
            events[e] = len(a) + len(b)
    return out, events


def test_stdp_off_or_zero_amplitudes_change_nothing():
    base = W.small(grid=2, M=40, K=25, seed=13, imposed_rate_hz=45.0, ext_rate_hz=2000.0)
    ref = oracle.OracleNet(base)
    ref.step(150)
    for cfg in (W.plastic(base, stdp_A_plus=0.0, stdp_A_minus=0.0, stdp_period_steps=50),):
        net = oracle.OracleNet(cfg)
        net.step(150)
        for a, b in zip(net.raster(), ref.raster()):
            assert np.array_equal(a, b)
        assert np.array_equal(net.csr()[1], ref.csr()[1])
        assert np.all(net.stdp()[0] == 0)


def test_stdp_changes_equal_the_pair_sum():
    cfg = _cfg(stdp_period_steps=10 ** 6)  # no application within the run
    T = 400
    net = oracle.OracleNet(cfg)
    net.step(T)
    delta, y, x = net.stdp()
    expect, events = _pair_sums(cfg, net, T)
    got = delta * 2.0 ** -16
    # each contribution is rounded once to 2^-16 mV; the traces carry float rounding
    tol = events * 2.0 ** -17 + 1e-5 * (np.abs(expect) + 0.01 * events)
    assert np.all(np.abs(got - expect) <= tol + 1e-12), np.max(np.abs(got - expect) - tol)
    plastic = events > 0
    assert plastic.sum() > 500 and np.count_nonzero(delta) > 500
    assert (expect > 0).sum() > 50 and (expect < 0).sum() > 50  # both signs occur
    M, n_exc = cfg["neurons_per_module"], oracle.constants(cfg)["n_exc"]
    rp = net.row_ptr()
    for i in range(net.N):  # inhibitory synapses never change
        if i % M >= n_exc:
            assert np.all(delta[int(rp[i]):int(rp[i + 1])] == 0)
    # the traces are the exponentially weighted spike counts
    st, ids = net.raster()
    for j in range(0, net.N, 7):
        b = st[ids == j].astype(np.float64)
        assert abs(y[j] - np.exp(-(T - 1 - b) / cfg["stdp_tau_minus_ms"]).sum()) < 1e-5
        assert abs(x[j] - np.exp(-(T - 1 - b) / cfg["stdp_tau_plus_ms"]).sum()) < 1e-5


def test_stdp_period_applies_the_clipped_change():
    cfg = _cfg(stdp_period_steps=300, stdp_w_max=0.31, stdp_A_plus=0.02, stdp_A_minus=0.021)
    T = 300
    net = oracle.OracleNet(cfg)
    w0 = net.csr()[1].copy()
    net.step(T)
    w1 = net.csr()[1]
    expect, events = _pair_sums(cfg, net, T)
    assert np.all(net.stdp()[0] == 0)  # accumulators restart after the application
    M, n_exc = cfg["neurons_per_module"], oracle.constants(cfg)["n_exc"]
    rp = net.row_ptr()
    exc = np.zeros(len(w0), bool)
    for i in range(net.N):
        exc[int(rp[i]):int(rp[i + 1])] = i % M < n_exc
    want = np.clip(w0 + expect, 0.0, np.float32(cfg["stdp_w_max"]))
    tol = events * 2.0 ** -17 + 1e-5 * (np.abs(expect) + 0.01 * events) + 1e-7
    assert np.all(np.abs(w1[exc] - want[exc]) <= tol[exc])
    assert np.array_equal(w1[~exc], w0[~exc])
    assert np.all((w1[exc] >= 0) & (w1[exc] <= np.float32(cfg["stdp_w_max"])))
    assert (w1[exc] == np.float32(cfg["stdp_w_max"])).sum() > 0  # the bound is reached
    # the new weights are what the next period delivers: the dynamics change
    net.step(200)
    ref = oracle.OracleNet(W.small(grid=2, M=40, K=25, seed=13, imposed_rate_hz=45.0, ext_rate_hz=2000.0))
    ref.step(T + 200)
    assert not np.array_equal(net.state()["V"], ref.state()["V"])
