"""The two-step spike exchange of the spatial decomposition (Sec. II-E) between
processes: gloo ranks on CPU, each owning one stripe of module rows.  The
spike lists are the oracle's raster of the whole network split by stripe; every
rank must receive, step by step, exactly the spikes of its peer stripes (the
stripes within the stencil's row radius), including steps with none."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _cfg(case):
    sys.path.insert(0, ROOT)
    from paper_1803_08833_gb300 import workloads as W
    if case == "gauss":  # radius 3: both stripes of a 2-way split are peers
        return W.small(grid=4, M=40, K=30, seed=5, imposed_rate_hz=60.0, ext_rate_hz=0.0)
    # cut-off of one grid step (radius 1) on 6 module rows: 3 stripes of 2 rows,
    # the outer stripes are not each other's peers
    return dict(W.small(grid=6, M=20, K=12, seed=6, imposed_rate_hz=40.0, ext_rate_hz=0.0), cutoff_um=100.0)


def _worker(rank, world, port, case, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1803_08833_gb300 import exchange as X
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        cfg = _cfg(case)
        WM = cfg["grid_w"] * cfg["neurons_per_module"]
        rows = [X.shard_rows(cfg["grid_h"], world, k) for k in range(world)]
        peer = X.peers(cfg, world, rank)
        net = oracle.OracleNet(cfg)
        steps = 40
        net.step(steps)
        st, ids = net.raster()
        got_steps = 0
        for t in range(steps):
            spk = ids[st == t]
            mine = spk[(spk >= rows[rank][0] * WM) & (spk < rows[rank][1] * WM)]
            if t % 7 == 3:
                mine = mine[:0]  # a step with no spikes on this rank
            recv = X.exchange_spikes(torch.from_numpy(mine.astype(np.int32)), peer)
            assert sorted(recv) == [q for q in peer if q != rank]
            for qr, buf in recv.items():
                exp = spk[(spk >= rows[qr][0] * WM) & (spk < rows[qr][1] * WM)]
                if t % 7 == 3:
                    exp = exp[:0]
                assert np.array_equal(buf.numpy().astype(np.uint32), exp), (rank, qr, t)
                got_steps += len(exp) > 0
        q.put((rank, peer, got_steps, None))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, None, 0, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("gauss", 2), ("short", 3)])
def test_two_step_exchange_between_gloo_ranks(case, world):
    import multiprocessing as mp
    sys.path.insert(0, ROOT)
    from paper_1803_08833_gb300 import exchange as X
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, peer, got, err in out:
        assert err is None, err
        assert got > 10  # the exchange carried spikes on most steps
    if case == "short":
        assert [o[1] for o in out] == [[0, 1], [0, 1, 2], [1, 2]]
    else:
        assert [o[1] for o in out] == [[0, 1], [0, 1]]
    assert X.stencil_row_radius(_cfg(case)) == (3 if case == "gauss" else 1)


def test_peer_relation_is_symmetric_and_local():
    sys.path.insert(0, ROOT)
    from paper_1803_08833_gb300 import exchange as X
    from paper_1803_08833_gb300 import workloads as W
    for cfg in (W.gauss_96x96_k1125(), W.exp_24x24_k2250(), dict(W.small(grid=9), cutoff_um=150.0)):
        R = X.stencil_row_radius(cfg)
        for n in (1, 2, 3, 5, 8):
            if n > cfg["grid_h"]:
                continue
            P = [set(X.peers(cfg, n, k)) for k in range(n)]
            for k in range(n):
                assert k in P[k]
                for j in range(n):
                    assert (j in P[k]) == (k in P[j])
                    a0, a1 = X.shard_rows(cfg["grid_h"], n, k)
                    b0, b1 = X.shard_rows(cfg["grid_h"], n, j)
                    gap = max(0, max(a0, b0) - min(a1, b1) + 1)  # rows between the stripes, plus one
                    assert (j in P[k]) == (gap <= R)
