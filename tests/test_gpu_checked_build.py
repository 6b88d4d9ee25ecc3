"""The checked build (-DSNN_CHECK, libsnn_check.so): device-side bounds checks
on the hot path's indexed writes (ring targets and slots, spike staging,
delay-window records), each of which sets an error bit and skips the access
instead of writing out of bounds.  Small parity cases run through it in a
child process (one library per process) in the per-step, persistent and
owner-windowed schedules and as a batch: every check passes, and the results
are the oracle's bit for bit."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import oracle
from paper_1803_08833_gb300 import snn, workloads as W
assert snn.LIB_PATH.endswith("libsnn_check.so")
cases = [W.small(grid=3, M=120, K=77, seed=5, imposed_rate_hz=30.0, ext_rate_hz=3000.0),
         W.pairwise(grid=3, M=90, seed=6, imposed_rate_hz=30.0),
         dict(W.small(grid=4, M=60, K=150, lateral="exp", seed=7, weight_dtype="bf16", imposed_rate_hz=35.0),
              table_layout="grouped")]
steps = 80
for cfg in cases:
    ref = oracle.OracleNet(cfg)
    ref.step(steps)
    rs, ri = ref.raster()
    for sched in (0, 2, 4):
        with snn.Network(cfg, raster_capacity=1 << 20) as net:
            net.set_schedule(sched)
            net.step(steps)
            st, ids = net.read_spikes()
            net.stats()  # raises if a device check failed
            assert np.array_equal(st, rs) and np.array_equal(ids, ri), sched
            assert np.array_equal(net.state()["ring"], ref.state()["ring"])
nets = [snn.Network(c, raster_capacity=1 << 20) for c in cases]
for n in nets:
    n.set_schedule(2)
with snn.Batch(nets) as b:
    b.step([steps] * len(nets))
for n, cfg in zip(nets, cases):
    ref = oracle.OracleNet(cfg)
    ref.step(steps)
    st, ids = n.read_spikes()
    n.stats()
    assert np.array_equal(st, ref.raster()[0]) and np.array_equal(ids, ref.raster()[1])
    n.close()
print("checked build ok")
"""


def test_checked_build_passes_every_bounds_check():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    sys.path.insert(0, ROOT)
    from paper_1803_08833_gb300 import _build
    _build.build(check=True)
    env = dict(os.environ, SNN_LIBRARY="check", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout
