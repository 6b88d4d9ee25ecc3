"""Spatial decomposition on one GPU: a network split into stripes of module rows
(Sec. II-D), each shard integrating its own neurons, the shards exchanging
their spikes (Sec. II-E) and arborizing the spikes they receive with their own
target-side copy of the synapses (Sec. II-C).  The union of the shards'
rasters, neuron states, delay rings and counters must equal the oracle's
undivided network bit for bit, for any number of shards."""
import numpy as np
import pytest

import oracle
from paper_1803_08833_gb300 import exchange as X
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


def _compare(st, ids, s, stats, ref):
    rs, ri = ref.raster()
    assert np.array_equal(st, rs) and np.array_equal(ids, ri), (len(st), len(rs))
    o = ref.state()
    assert np.array_equal(s["V"].view(np.uint32), o["V"].view(np.uint32))
    assert np.array_equal(s["c"].view(np.uint32), o["c"].view(np.uint32))
    assert np.array_equal(s["ref"], o["ref"])
    assert np.array_equal(s["ring"], o["ring"])
    b = ref.stats()
    assert stats["n_spikes"] == b["spikes"] and stats["rec_events"] == b["rec_events"]
    assert stats["ext_events"] == b["ext_events"]
    return len(st)


CASES = {
    "gauss": (lambda: W.small(grid=6, M=100, K=150, seed=21, imposed_rate_hz=30.0, ext_rate_hz=3000.0), 120),
    "exp_bf16": (lambda: dict(W.small(grid=5, M=80, K=200, lateral="exp", seed=22, weight_dtype="bf16",
                                      imposed_rate_hz=35.0), grid_h=7), 100),
    "short_cutoff_ragged": (lambda: dict(W.small(grid=5, M=77, K=37, seed=23, imposed_rate_hz=40.0),
                                         grid_h=9, cutoff_um=120.0), 100),
    "silent_spec": (lambda: W.gauss_4x4_k1000(seed=2), 300),
}


@pytest.mark.parametrize("n_shards", [1, 2, 3, 4])
@pytest.mark.parametrize("name", sorted(CASES))
def test_union_of_shards_equals_oracle(snn, name, n_shards):
    make, steps = CASES[name]
    cfg = make()
    if n_shards > cfg["grid_h"]:
        pytest.skip("more shards than module rows")
    ref = oracle.OracleNet(cfg)
    ref.step(steps)
    with snn.ShardedNetwork(cfg, n_shards, raster_capacity=1 << 20) as net:
        infos = [sh.info() for sh in net.shards]
        # the stripes tile the neurons; every synapse sits in exactly one shard's table
        assert infos[0]["n0"] == 0 and infos[-1]["n1"] == ref.N
        assert all(a["n1"] == b["n0"] for a, b in zip(infos, infos[1:]))
        assert sum(i["table_synapses"] for i in infos) == ref.N * cfg["K"]
        for k, i in enumerate(infos):  # the library's peers are the exchange module's
            assert list(range(i["peer_lo"], i["peer_hi"] + 1)) == X.peers(cfg, n_shards, k)
        net.step(steps // 2)
        net.step(steps - steps // 2)
        st, ids = net.read_spikes()
        n = _compare(st, ids, net.state(), net.stats(), ref)
    if "silent" not in name:
        assert n > 500


def test_exchange_through_separate_receive_buffers(snn):
    """The multi-process form, on one device: after each shard integrates, the
    peers' spike counts are read first and then exactly that many ids are
    copied into receive buffers of the receiving shard (what the two-step
    message exchange delivers); each shard arborizes its own outbox and the
    received buffers."""
    import torch
    cfg = CASES["gauss"][0]()
    n, steps = 3, 60
    ref = oracle.OracleNet(cfg)
    ref.step(steps)
    shards = [snn.Shard(cfg, n, k, raster_capacity=1 << 20) for k in range(n)]
    peers = [X.peers(cfg, n, k) for k in range(n)]
    recv = {(k, q): (torch.empty(cfg["grid_w"] * cfg["grid_h"] * cfg["neurons_per_module"], dtype=torch.int32,
                                 device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda"))
            for k in range(n) for q in peers[k] if q != k}
    try:
        views = [sh.outbox_tensors() for sh in shards]
        for t in range(steps):
            for sh in shards:
                sh.integrate()
            # step 1: the counts; step 2: exactly that many ids into the receive buffers
            cnt = [int(c.item()) for _, c in views]
            for (k, q), (buf, c) in recv.items():
                buf[:cnt[q]].copy_(views[q][0][:cnt[q]])
                c.fill_(cnt[q])
            for k, sh in enumerate(shards):
                lists = [sh.outbox()] + [(recv[(k, q)][0].data_ptr(), recv[(k, q)][1].data_ptr())
                                         for q in peers[k] if q != k]
                sh.deliver(lists)
        torch.cuda.synchronize()
        parts = [sh.read_spikes() for sh in shards]
        st = np.concatenate([p[0] for p in parts])
        ids = np.concatenate([p[1] for p in parts])
        o = np.lexsort((ids, st))
        states = [sh.state() for sh in shards]
        s = {k: np.concatenate([x[k] for x in states], axis=1 if k == "ring" else 0) for k in ("V", "c", "ref", "ring")}
        stats = {}
        for sh in shards:
            for key, v in sh.stats().items():
                stats[key] = stats.get(key, 0) + v
        assert _compare(st[o], ids[o], s, stats, ref) > 500
    finally:
        for sh in shards:
            sh.close()


def test_shard_argument_errors(snn):
    with pytest.raises(snn.SnnError, match="fixed out-degree"):
        snn.Shard(W.pairwise(grid=3, M=30), 2, 0)
    with pytest.raises(snn.SnnError, match="index"):
        snn.Shard(W.small(grid=3), 4, 0)  # more shards than module rows
    with pytest.raises(snn.SnnError, match="index"):
        snn.Shard(W.small(grid=3), 2, 2)
