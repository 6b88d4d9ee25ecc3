"""Pin the oracle's FP64 reference mode (Eq. 1-2 and the delay queues of
Sec. II-A in double precision, no fixed point).  This is the reference of the
BF16 precision claim, so it is pinned as tightly as the FP32 mode: the
single-neuron update against closed forms and an ODE solution, and the
network loop (initial state, drive, step order, ring) against trajectories
rebuilt from that update and from sums of the FP64 weights."""
import math

import numpy as np
import pytest

import oracle
from paper_1803_08833_gb300 import workloads as W


def _cfg(**kw):
    c = W.small()
    c.update(kw)
    return c


def _isi64(cfg, J, n_max=4000):
    """Steps between two spikes under a constant input of J mV per step."""
    k = oracle.constants(cfg)
    V, c, ref = cfg["V_reset_mV"], 0.0, k["ref_steps"]  # state right after a spike
    for n in range(1, n_max):
        V, c, ref, s = oracle.lif_update64(cfg, V, c, ref, True, J)
        if s:
            return n
    return None


def test_fp64_discrete_f_I_closed_form():
    """Adaptation off, constant jump J: V_n = V_inf + (V_r - V_inf) a^n with
    V_inf = J / (1 - a); the interspike interval is the refractory steps plus
    the first n with V_n > V_th, exactly (double precision, away from ties)."""
    cfg = _cfg(alpha_c=0.0)
    a = math.exp(-cfg["dt_ms"] / cfg["tau_m_ms"])
    Vr, Vth = cfg["V_reset_mV"], cfg["V_th_mV"]
    checked = 0
    for J in np.linspace(1.0, 6.0, 157):
        Vinf = J / (1 - a)
        if Vinf <= Vth:
            assert _isi64(cfg, J, 600) is None
            continue
        n = 1
        while Vinf + (Vr - Vinf) * a ** n <= Vth:
            n += 1
        margin = min(abs(Vinf + (Vr - Vinf) * a ** m - Vth) for m in (n - 1, n))
        if margin < 1e-9:
            continue
        assert _isi64(cfg, J) == n + 2, J
        checked += 1
    assert checked > 100


def test_fp64_free_trajectory_is_the_geometric_closed_form():
    """Below threshold the membrane under a constant J follows the closed form
    to double rounding over hundreds of steps (a wrong a_m or a dropped term
    would drift)."""
    cfg = _cfg(alpha_c=0.0, V_th_mV=1e9)
    a = math.exp(-cfg["dt_ms"] / cfg["tau_m_ms"])
    for J in (0.37, 1.9, -0.8):
        V, c, ref = 3.0, 0.0, 0
        Vinf = J / (1 - a)
        for n in range(1, 400):
            V, c, ref, s = oracle.lif_update64(cfg, V, c, ref, True, J)
            assert abs(V - (Vinf + (3.0 - Vinf) * a ** n)) < 1e-11 * max(1.0, abs(Vinf)), (J, n)


def test_fp64_propagator_matches_ode_solution():
    """One free step equals the solution of dV/dt = -(V-E)/tau_m - g_c c,
    dc/dt = -c/tau_c over dt (numerical, rtol 1e-12), plus the step's jump."""
    from scipy.integrate import solve_ivp
    for E in (0.0, -3.5, 2.25):
        for tc in (500.0, 20.0, 7.0):  # tau_c = tau_m takes the degenerate branch
            cfg = _cfg(E_mV=E, tau_c_ms=tc)
            tm, gc, dt = cfg["tau_m_ms"], cfg["g_c_mV"], cfg["dt_ms"]
            for V0, c0, I in ((12.0, 0.0, 0.0), (5.0, 0.7, 0.0), (-4.0, 2.5, 0.61), (18.0, 0.3, -0.137)):
                sol = solve_ivp(lambda t, y: [-(y[0] - E) / tm - gc * y[1], -y[1] / tc], (0, dt),
                                [V0, c0], rtol=1e-12, atol=1e-14, method="DOP853")
                V, c, ref, s = oracle.lif_update64(cfg, V0, c0, 0, True, I)
                assert not s
                assert abs(V - (sol.y[0, -1] + I)) < 1e-9 * max(1.0, abs(V)), (E, tc, V0, c0)
                assert abs(c - sol.y[1, -1]) < 1e-11 * max(1.0, c0)


def test_fp64_constants_against_the_ode():
    """kc is the drop of V over dt caused by c = 1 (V = E, no input), a_c the
    decay of c: both from the ODE solution, for tau_c != tau_m and = tau_m."""
    from scipy.integrate import solve_ivp
    for tc in (500.0, 20.0):
        cfg = _cfg(tau_c_ms=tc)
        tm, gc, dt = cfg["tau_m_ms"], cfg["g_c_mV"], cfg["dt_ms"]
        k = oracle.constants64(cfg)
        sol = solve_ivp(lambda t, y: [-y[0] / tm - gc * y[1], -y[1] / tc], (0, dt), [0.0, 1.0],
                        rtol=1e-13, atol=1e-15, method="DOP853")
        assert abs(-sol.y[0, -1] - k["kc"]) < 1e-10
        assert abs(sol.y[1, -1] - k["a_c"]) < 1e-12
        assert k["a_m"] == math.exp(-dt / tm)


def test_fp64_reset_rules():
    cfg = _cfg()
    k = oracle.constants(cfg)
    kk = oracle.constants64(cfg)
    # refractory: input discarded, V held, c keeps decaying, earliest next spike 3 steps on
    V, c, ref, s = oracle.lif_update64(cfg, 19.0, 0.5, 0, True, 10.0)
    assert s and V == cfg["V_reset_mV"] and ref == k["ref_steps"] == 2
    assert c == 0.5 * kk["a_c"] + float(np.float32(cfg["alpha_c"]))  # parameters are float32
    for r in (1, 0):
        c_prev = c
        V, c, ref, s = oracle.lif_update64(cfg, V, c, ref, True, 100.0)
        assert not s and V == cfg["V_reset_mV"] and ref == r and c == c_prev * kk["a_c"]
    V, c, ref, s = oracle.lif_update64(cfg, V, c, ref, True, 100.0)
    assert s
    # strict threshold at the fixed point V = E = V_th
    cfg2 = _cfg(E_mV=20.0)
    V, c, ref, s = oracle.lif_update64(cfg2, 20.0, 0.0, 0, True, 0.0)
    assert V == 20.0 and not s
    V, c, ref, s = oracle.lif_update64(cfg2, 20.0, 0.0, 0, True, 1e-12)
    assert s
    # no adaptation for inhibitory neurons; forced spikes obey the refractory period
    V, c, ref, s = oracle.lif_update64(cfg, 19.9, 0.0, 0, False, 2.0)
    assert s and c == 0.0
    V, c, ref, s = oracle.lif_update64(cfg, 0.0, 0.0, 0, True, 0.0, forced=True)
    assert s and ref == 2
    V, c, ref, s = oracle.lif_update64(cfg, V, c, ref, True, 0.0, forced=True)
    assert not s


def test_fp64_network_loop_rebuilt_from_the_update():
    """K = 0 (external drive and forced spikes only): the FP64 network equals,
    bit for bit, the trajectories rebuilt neuron by neuron from the initial
    state (V0 = V_th U[0,1) of Philox (i, 0, INIT)), the drive draws and the
    single-neuron update."""
    cfg = W.small(grid=2, M=50, K=0, seed=21, ext_rate_hz=4000.0, imposed_rate_hz=20.0)
    T = 250
    net = oracle.OracleNet(cfg, fp64=True)
    net.step(T)
    st = net.state()
    rs, ri = net.raster()
    seed = cfg["seed"]
    key = (seed & 0xFFFFFFFF, seed >> 32)
    M, n_exc = cfg["neurons_per_module"], oracle.constants(cfg)["n_exc"]
    J = float(np.float32(cfg["J_ext_mV"]))
    spikes = []
    for i in range(net.N):
        u0 = oracle.philox([i, 0, 2, 0], key)[0]
        V = float(np.float32(cfg["V_th_mV"])) * ((u0 >> 8) * 2.0 ** -24)
        c, ref = 0.0, 0
        for t in range(T):
            n_ext, forced = oracle.drive(cfg, i, t)
            V, c, ref, s = oracle.lif_update64(cfg, V, c, ref, (i % M) < n_exc, n_ext * J, forced)
            if s:
                spikes.append((t, i))
        assert V == st["V"][i] and c == st["c"][i] and ref == st["ref"][i], i
    spikes.sort()
    assert len(spikes) == len(rs) > 50
    assert all(a == (int(x), int(y)) for a, x, y in zip(spikes, rs, ri))


def test_fp64_ring_delivers_the_fp64_weights_at_the_delay():
    """One excitatory spike into a quiet network (no drive, V = c = 0 elsewhere,
    E = 0): each target's V follows V_s = V_{s-1} a_m + (sum of the FP64
    weights of its synapses with delay s), in the oracle's summation order,
    and nothing else moves."""
    cfg = W.small(grid=3, M=60, K=40, seed=17, ext_rate_hz=0.0, E_mV=0.0)
    net = oracle.OracleNet(cfg, fp64=True)
    N = net.N
    V0 = np.zeros(N)
    V0[7] = 25.0  # above threshold: neuron 7 (excitatory) spikes at step 0
    net.set_state(V=V0, c=np.zeros(N))
    tgt, w, d = net.csr()
    rp = net.row_ptr()
    row = slice(int(rp[7]), int(rp[8]))
    T = int(d[row].max()) + 3
    a_m = oracle.constants64(cfg)["a_m"]
    expect = np.zeros(N)
    for s in range(T):
        net.step(1)
        arr = np.zeros(N)
        for k in range(row.start, row.stop):  # the oracle's order: synapse by synapse
            if s >= 1 and d[k] == s:
                arr[tgt[k]] += w[k]
        expect = expect * a_m + arr
        if s == 0:
            expect[7] = cfg["V_reset_mV"]
        elif s <= 2:
            expect[7] = cfg["V_reset_mV"]  # refractory
        got = net.state()["V"]
        assert np.array_equal(got[np.arange(N) != 7], expect[np.arange(N) != 7]), s
    rs, ri = net.raster()
    assert list(zip(rs.tolist(), ri.tolist())) == [(0, 7)]
    assert np.all(net.state()["ring"] == 0.0)
    assert w.dtype == np.float64 and np.all((w[row] >= 0.1) & (w[row] < 0.3))
