"""Pin the oracle's connectivity (lateral kernels of Sec. I / Sec. III-B,
synapse generation of Sec. II-B) against closed forms, brute-force enumeration
and chi-square tests."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1803_08833_gb300 import workloads as W


def _kernel(cfg, d2):
    s = cfg["spacing_um"]
    if cfg["kernel"] == "gauss":
        return math.exp(-(d2 * s * s) / (2 * cfg["sigma_um"] ** 2))
    return math.exp(-s * math.sqrt(d2) / cfg["lambda_um"])


def _stencil(R2):
    R = int(math.isqrt(R2))
    return [(dx, dy) for dy in range(-R, R + 1) for dx in range(-R, R + 1) if dx * dx + dy * dy <= R2]


def test_stencil_sizes():
    """3 sigma at 100 um spacing keeps r^2 <= 9 grid units (29 modules); 1.2 mm
    keeps r^2 <= 144 (441 modules): lattice-point counts of the two discs."""
    g = W.gauss_4x4_k1000()
    e = W.exp_24x24_k2250()
    assert oracle.constants(g)["R2"] == 9 and oracle.constants(g)["max_offsets"] == 29
    assert oracle.constants(e)["R2"] == 144 and oracle.constants(e)["max_offsets"] == 441
    assert len(_stencil(9)) == 29 and len(_stencil(144)) == 441
    # interior source of a 24x24 grid sees the whole disc; a corner sees a quarter
    e2 = dict(e)
    T, TM, p = oracle.cdf_table(dict(g, grid_w=24, grid_h=24), 12 * 24 + 12)
    assert len(T) == 29
    T, TM, p = oracle.cdf_table(e2, 0)
    assert len(T) == sum(1 for dx, dy in _stencil(144) if dx >= 0 and dy >= 0)


@pytest.mark.parametrize("lateral", ["gauss", "exp"])
def test_two_by_two_brute_force(lateral):
    """On a 2x2 grid every source sees all four modules (d2 = 0, 1, 1, 2); the
    table's probability mass equals the normalised kernel written out directly."""
    cfg = W.small(grid=2, lateral=lateral)
    for s in range(4):
        T, TM, p = oracle.cdf_table(cfg, s)
        assert len(T) == 4 and sorted(TM.tolist()) == [0, 1, 2, 3]
        sx, sy = s % 2, s // 2
        f = [_kernel(cfg, (m % 2 - sx) ** 2 + (m // 2 - sy) ** 2) for m in TM.tolist()]
        p_direct = np.array(f) / sum(f)
        assert np.allclose(p, p_direct, rtol=1e-14, atol=0)
        edges = np.concatenate([[0], T[:-1].astype(np.int64), [2 ** 32]])
        mass = np.diff(edges)
        assert np.all(np.abs(mass - p_direct * 2 ** 32) <= 1.0)


@pytest.mark.parametrize("lateral", ["gauss", "exp"])
def test_two_by_two_empirical_frequencies(lateral):
    cfg = W.small(grid=2, M=50, K=400, lateral=lateral, seed=11)
    net = oracle.OracleNet(cfg)
    tgt, w, d = net.csr()
    M, K = 50, 400
    src_mod = np.repeat(np.arange(net.N) // M, K)
    tgt_mod = tgt // M
    for s in range(4):
        _, TM, p = oracle.cdf_table(cfg, s)
        obs = np.bincount(tgt_mod[src_mod == s], minlength=4)[TM]
        chi = stats.chisquare(obs, p * obs.sum())
        assert chi.pvalue > 1e-3, (s, obs, p)


def test_total_synapses_and_ranges():
    cfg = W.gauss_4x4_k1000(seed=2)
    net = oracle.OracleNet(cfg)
    tgt, w, d = net.csr()
    N, K, M = 16000, 1000, 1000
    assert len(tgt) == N * K == net.N * net.K
    assert tgt.max() < N
    src = np.repeat(np.arange(N), K)
    exc = (src % M) < 800
    we, de = w[exc], d[exc]
    assert we.min() >= np.float32(0.1) and we.max() <= np.float32(0.3)  # float rounding may reach 0.3f
    assert abs(we.astype(np.float64).mean() - 0.2) < 4 * (0.2 / math.sqrt(12)) / math.sqrt(we.size)
    assert np.all(w[~exc] == np.float32(-0.8)) and np.all(d[~exc] == 1)
    assert de.min() == 1 and de.max() == 20
    chi = stats.chisquare(np.bincount(de, minlength=21)[1:])
    assert chi.pvalue > 1e-3
    # every target lies within the cut-off radius of its source module
    sm, tm = src // M, tgt // M
    d2 = (sm % 4 - tm % 4) ** 2 + (sm // 4 - tm // 4) ** 2
    assert d2.max() <= 9
    # target neuron uniform within its module (uniform in-degree over positions)
    chi = stats.chisquare(np.bincount(tgt % M, minlength=M))
    assert chi.pvalue > 1e-3


@pytest.mark.parametrize("lateral,grid,seeds", [("gauss", 9, (1, 2, 3, 4, 5)), ("exp", 27, (1, 2, 3))])
def test_distance_histogram_matches_kernel(lateral, grid, seeds):
    """Distances drawn from interior sources follow the normalised kernel."""
    R2 = 9 if lateral == "gauss" else 144
    R = int(math.isqrt(R2))
    for seed in seeds:
        cfg = W.small(grid=grid, M=8, K=300 if lateral == "gauss" else 120, lateral=lateral, seed=seed)
        net = oracle.OracleNet(cfg)
        tgt, _, _ = net.csr()
        M, K = 8, cfg["K"]
        src = np.repeat(np.arange(net.N) // M, K)
        sx, sy = src % grid, src // grid
        interior = (sx >= R) & (sx < grid - R) & (sy >= R) & (sy < grid - R)
        tm = tgt // M
        d2 = (tm % grid - sx) ** 2 + (tm // grid - sy) ** 2
        d2 = d2[interior]
        values = sorted({dx * dx + dy * dy for dx, dy in _stencil(R2)})
        mult = {v: sum(1 for dx, dy in _stencil(R2) if dx * dx + dy * dy == v) for v in values}
        f = np.array([mult[v] * _kernel(cfg, v) for v in values])
        p = f / f.sum()
        obs = np.array([(d2 == v).sum() for v in values])
        chi = stats.chisquare(obs, p * obs.sum())
        assert chi.pvalue > 1e-3, (seed, chi.pvalue)


def test_bf16_weights_are_round_to_nearest_even():
    import torch
    cfg32 = W.small(grid=2, M=40, K=50, seed=5)
    cfg16 = dict(cfg32, weight_dtype="bf16")
    _, w32, d32 = oracle.OracleNet(cfg32).csr()
    t16, w16, d16 = oracle.OracleNet(cfg16).csr()
    ref = torch.from_numpy(w32).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(w16, ref)
    assert np.array_equal(d16, d32)
    assert not np.array_equal(w16, w32)


def test_seed_changes_draws_and_same_seed_repeats():
    a = oracle.OracleNet(W.small(seed=1)).csr()[0]
    b = oracle.OracleNet(W.small(seed=1)).csr()[0]
    c = oracle.OracleNet(W.small(seed=2)).csr()[0]
    assert np.array_equal(a, b) and not np.array_equal(a, c)
