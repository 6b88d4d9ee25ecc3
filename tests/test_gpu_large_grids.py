"""Table I's larger grids (48x48: 2.88 M neurons, 96x96: 11.5 M neurons) against
the oracle, step by step, with the banded delivery at its full geometry.

The oracle cannot simulate these networks in test time, so each GPU step is
checked against the oracle's restatement of that one step, from the GPU's
state before it:
  - the whole delay ring after the step equals the ring before it, with the
    consumed slot cleared, plus the fixed-point weight of every synapse of
    every neuron that spiked in the step, at row (t + delay) mod D, the rows
    drawn by the oracle's own generator;
  - V, c and the refractory counter of 3,000 sampled neurons equal the
    oracle's update of their previous state with the consumed ring slot and
    their external drive, and they spike exactly when the oracle says so.
Every step is one persistent launch (schedule 2) whose delivery runs in the
default number of bands: the target module rows split so that one band's ring
columns stay in L2 (4 bands at 48x48 and 13 at 96x96 on a GB300).
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


def _step_by_step(snn, cfg, steps, min_bands, warm=2, n_sample=3000, seed=0, schedule=2):
    rng = np.random.default_rng(seed)
    k = oracle.constants(cfg)
    M = cfg["neurons_per_module"]
    scale = float(2 ** cfg["fx_shift"])
    with snn.Network(cfg, raster_capacity=1 << 24) as net:
        bands = net.set_bands(0)
        assert bands >= min_bands, bands
        net.set_schedule(schedule)
        N, D = net.N, net.D
        sample = np.unique(np.concatenate([rng.integers(0, N, n_sample), [0, M - 1, N // 2, N - 1]]))
        exc = (sample % M) < k["n_exc"]
        net.step(warm)
        prev = net.state()
        checked_spikes = 0
        for t in range(warm, warm + steps):
            net.clear_raster()
            ev0 = net.stats()["rec_events"]
            net.step(1)
            cur = net.state()
            st, ids = net.read_spikes()
            assert np.all(st == t) and np.all(np.diff(ids.astype(np.int64)) > 0)
            slot = t % D
            # the sampled neurons: one oracle update from the previous state
            spiked = set(ids.tolist())
            for j, i in enumerate(sample.tolist()):
                n_ext, forced = oracle.drive(cfg, i, t)
                I = int(prev["ring"][slot, i]) + n_ext * k["J_ext_fx"]
                V, c, ref, sp = oracle.lif_update(cfg, float(prev["V"][i]), float(prev["c"][i]),
                                                  int(prev["ref"][i]), bool(exc[j]), I, forced)
                assert np.float32(V) == cur["V"][i] and np.float32(c) == cur["c"][i] and ref == cur["ref"][i], (t, i)
                assert sp == (i in spiked), (t, i)
                checked_spikes += sp
            # the whole ring: previous ring, consumed slot cleared, plus every spiker's row
            tgt, w, d, ln = oracle.gen_rows_list(cfg, ids)
            assert int(ln.sum()) == net.stats()["rec_events"] - ev0
            flat = ((t + d.astype(np.int64)) % D) * N + tgt.astype(np.int64)
            add = np.bincount(flat, weights=np.rint(w.astype(np.float64) * scale), minlength=D * N)
            expect = prev["ring"].astype(np.int64)
            expect[slot] = 0
            expect += add.reshape(D, N).astype(np.int64)
            del add, flat
            assert np.array_equal(cur["ring"].astype(np.int64), expect), t
            del expect
            prev = cur
        return bands, checked_spikes


def test_48x48_fixed_law_banded_steps_equal_oracle(snn):
    cfg = W.gauss_48x48_k1125(seed=6, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ, table_layout="grouped")
    bands, sp = _step_by_step(snn, cfg, steps=4, min_bands=2)
    print("\n48x48 fixed law: %d bands, %d sampled spikes checked" % (bands, sp))


def test_48x48_fixed_law_pulled_windows_steps_equal_oracle(snn):
    """Schedule 5 at 2.88 M neurons: bands of 14-16 modules (20,000 neurons),
    so only 2 steps of window fit in shared memory and most events take the
    far path through the ring; every step still equals the oracle's."""
    cfg = W.gauss_48x48_k1125(seed=9, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ, table_layout="grouped")
    _, sp = _step_by_step(snn, cfg, steps=4, min_bands=1, schedule=5)
    print("\n48x48 fixed law, schedule 5: %d sampled spikes checked" % sp)


def test_48x48_pairwise_law_banded_steps_equal_oracle(snn):
    cfg = W.pairwise(grid=48, seed=7, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ)
    bands, sp = _step_by_step(snn, cfg, steps=3, min_bands=2)
    print("\n48x48 per-pair law: %d bands, %d sampled spikes checked" % (bands, sp))


def test_96x96_fixed_law_banded_steps_equal_oracle(snn):
    """11.5 M neurons, 12.96 G synapses (104 GB of table), the ring (968 MB)
    eight times the L2: 13 bands on a GB300."""
    cfg = W.gauss_96x96_k1125(seed=8, imposed_rate_hz=W.PAPER_RATE_GAUSS_HZ, table_layout="grouped")
    with snn.Network(cfg, raster_capacity=1 << 10) as net:  # a band of 76,000 neurons: no window row fits
        with pytest.raises(snn.SnnError, match="does not fit in shared memory"):
            net.set_schedule(5)
    bands, sp = _step_by_step(snn, cfg, steps=2, min_bands=8)
    print("\n96x96 fixed law: %d bands, %d sampled spikes checked" % (bands, sp))
