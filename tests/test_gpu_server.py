"""Serving: requests admitted under a memory budget into a continuous-batching
loop.  Every result must be the same alone and in the mix (bit for bit: the
spike raster and final state hashes), and match the oracle."""
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


def _fnv(arrs):
    h = 1469598103934665603
    for a in arrs:
        for b in np.ascontiguousarray(a).view(np.uint8).tolist():
            h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


REQUESTS = [
    (W.small(grid=2, M=120, K=77, seed=5, imposed_rate_hz=30.0, ext_rate_hz=3000.0), 90),
    (W.small(grid=3, M=100, K=200, lateral="exp", seed=6, weight_dtype="bf16", imposed_rate_hz=35.0), 140),
    (W.small(grid=4, M=50, K=150, seed=7, ext_rate_hz=5000.0), 60),
    (dict(W.small(grid=3, M=333, K=37, seed=9, imposed_rate_hz=40.0), grid_h=2), 250),
    (W.small(grid=2, M=64, K=10, seed=1, ext_rate_hz=0.0), 30),
]


def _serve(snn, reqs, budget, chunk=40, stagger=False):
    out = {}
    with snn.Server(budget, chunk_steps=chunk) as srv:
        ids = []
        for k, (cfg, steps) in enumerate(reqs):
            ids.append(srv.submit(cfg, steps))
            if stagger and k % 2 == 1:
                srv.tick()  # later requests arrive while earlier ones run
        for _ in range(1000):
            a, q = srv.tick()
            for r in srv.poll():
                out[r["request_id"]] = r
            if a == 0 and q == 0:
                break
        for r in srv.poll():
            out[r["request_id"]] = r
    return [out[i] for i in ids]


def test_results_alone_equal_results_in_the_mix(snn):
    budget = 8 << 30
    alone = [_serve(snn, [r], budget)[0] for r in REQUESTS]
    mixed = _serve(snn, REQUESTS, budget, stagger=True)
    for a, m in zip(alone, mixed):
        assert a["status"] == 0 and m["status"] == 0
        for k in ("steps", "n_spikes", "rec_events", "ext_events", "raster_hash", "state_hash"):
            assert a[k] == m[k], k
    # one of them against the oracle
    cfg, steps = REQUESTS[1]
    ref = oracle.OracleNet(cfg)
    ref.step(steps)
    st, ids = ref.raster()
    assert mixed[1]["n_spikes"] == len(st) == ref.stats()["spikes"]
    assert mixed[1]["raster_hash"] == _fnv([st, ids])
    assert mixed[1]["state_hash"] == _fnv([ref.state()["V"]])


def test_budget_admission_queues_and_rejects(snn):
    need = [snn.estimate_bytes(c, 1 << 16) for c, _ in REQUESTS]
    budget = int(sum(sorted(need)[-2:]) * 1.01)  # room for two of the largest at a time
    res = _serve(snn, REQUESTS, budget, chunk=25)
    assert all(r["status"] == 0 for r in res)
    assert max(r["queue_ms"] for r in res) > 0.0
    with snn.Server(need[0] // 2) as srv:
        with pytest.raises(snn.SnnError, match="SNN_EBUDGET"):
            srv.submit(REQUESTS[0][0], 10)


def test_pairwise_requests_in_the_mix(snn):
    """Requests under the per-pair law (variable-length rows) served together
    with fixed out-degree ones: the same alone and in the mix, and a pairwise
    result equal to the oracle."""
    reqs = [(W.pairwise(grid=4, M=80, seed=21, imposed_rate_hz=25.0), 70),
            REQUESTS[0],
            (W.pairwise(grid=6, M=40, lateral="exp", seed=22, weight_dtype="bf16", imposed_rate_hz=35.0), 110)]
    budget = 8 << 30
    alone = [_serve(snn, [r], budget)[0] for r in reqs]
    mixed = _serve(snn, reqs, budget, stagger=True)
    for a, m in zip(alone, mixed):
        assert a["status"] == 0 and m["status"] == 0
        for k in ("steps", "n_spikes", "rec_events", "ext_events", "raster_hash", "state_hash"):
            assert a[k] == m[k], k
    cfg, steps = reqs[0]
    ref = oracle.OracleNet(cfg)
    ref.step(steps)
    st, ids = ref.raster()
    assert mixed[0]["n_spikes"] == len(st) and mixed[0]["rec_events"] == ref.stats()["rec_events"]
    assert mixed[0]["raster_hash"] == _fnv([st, ids])
    assert mixed[0]["state_hash"] == _fnv([ref.state()["V"]])


def test_server_batch_layout_changes_no_result(snn):
    """Every tick's batch in the global layout, launch shape 1, a small ring
    budget: each request's result equals the default layout's."""
    import paper_1803_08833_gb300.workloads as W
    reqs = [(W.small(grid=2, M=120, K=77, seed=5, imposed_rate_hz=30.0), 90),
            (W.small(grid=3, M=80, K=150, lateral="exp", seed=6, imposed_rate_hz=35.0), 140),
            (W.small(grid=2, M=64, K=30, seed=7, imposed_rate_hz=20.0), 60)]
    out = []
    for layout in (None, ("global", 1, 1 << 20)):
        with snn.Server(1 << 32, chunk_steps=25, max_slots=8) as srv:
            if layout:
                srv.set_batch(*layout)
            for cfg, steps in reqs:
                srv.submit(cfg, steps, raster_capacity=1 << 16)
            res = []
            while len(res) < len(reqs):
                srv.tick()
                res += srv.poll()
            out.append(sorted((r["request_id"], r["raster_hash"], r["state_hash"], r["n_spikes"]) for r in res))
    assert out[0] == out[1]
    assert all(r[3] > 0 for r in out[0])
