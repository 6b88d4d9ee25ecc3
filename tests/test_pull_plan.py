"""Host logic of schedule 5 (no GPU): the bands every SM owns and, per band,
the runs it pulls -- for each source module whose stencil reaches the band,
the stencil entries [j0, j1) whose target modules overlap the band.  Checked
against brute force over every (source module, stencil entry), with the
stencil of each source module taken from the oracle's target tables (so the
library's stencil order is pinned to the oracle's, too)."""
import numpy as np
import pytest

import oracle
from paper_1803_08833_gb300 import workloads as W


@pytest.fixture(scope="module")
def snn():
    from paper_1803_08833_gb300 import _build
    from paper_1803_08833_gb300 import snn as S
    _build.build()
    S.load()
    return S


CASES = {
    "gauss_24x24_M1250": W.gauss_24x24_k1125(seed=1),
    # the per-pair law: its rows number every stencil offset, out-of-grid ones as empty segments
    "pairwise_gauss_12x12_M1250": W.pairwise(grid=12, seed=1),
    "pairwise_exp_5x7_M90": dict(W.pairwise(grid=5, M=90, lateral="exp", seed=2), grid_h=7),
    "exp_6x6_M120": W.small(grid=6, M=120, K=400, lateral="exp", seed=5),
    "ragged_3x2_M333": dict(W.small(grid=3, M=333, K=37, seed=9), grid_h=2),
    "short_cutoff_7x9_M77": dict(W.small(grid=7, M=77, K=60, seed=12), grid_h=9, cutoff_um=120.0),
    "spec_4x4_M1000": W.gauss_4x4_k1000(seed=1),
    # one module: every band's runs come from it alone
    "single_module_1x1_M50": W.small(grid=1, M=50, K=20, seed=3),
    # the per-pair law with modules split inside quads
    "pairwise_ragged_3x4_M43": dict(W.pairwise(grid=3, M=43, seed=7), grid_h=4),
}


def _entry_modules(cfg, s):
    """Target module of every segment-index entry of source module s (-1: an
    out-of-grid entry, an empty segment): the fixed law's entries are its
    in-grid stencil modules (the oracle's target table), the per-pair law's
    are all offsets of the oracle's pair stencil."""
    if cfg.get("conn_rule") == "pairwise":
        gw, gh = cfg["grid_w"], cfg["grid_h"]
        dx, dy = oracle.pair_stencil(cfg)[:2]
        tx, ty = s % gw + dx, s // gw + dy
        inside = (tx >= 0) & (ty >= 0) & (tx < gw) & (ty < gh)
        return np.where(inside, ty * gw + tx, -1)
    return np.asarray(oracle.cdf_table(cfg, s)[1]).astype(np.int64)


def _brute_runs(cfg, n0, n1):
    """Runs of the band of neurons [n0, n1): (source module, j0, j1), the
    entries from the first to the last whose target module the band touches."""
    M = cfg["neurons_per_module"]
    nm = cfg["grid_w"] * cfg["grid_h"]
    m_lo, m_hi = n0 // M, (n1 - 1) // M
    out = []
    for s in range(nm):
        TM = _entry_modules(cfg, s)
        hit = np.nonzero((TM >= m_lo) & (TM <= m_hi))[0]
        if len(hit) == 0:
            continue
        j0, j1 = int(hit[0]), int(hit[-1]) + 1
        inner = TM[j0:j1]
        # in between only the band's modules, or empty segments
        assert np.all((inner == -1) | ((inner >= m_lo) & (inner <= m_hi))), "non-contiguous entries"
        out.append((s, j0, j1))
    return out


@pytest.mark.parametrize("sms", [152, 7, 1, 1000])
@pytest.mark.parametrize("band_mode", [1, 2])
@pytest.mark.parametrize("name", sorted(CASES))
def test_bands_and_runs_equal_brute_force(snn, name, band_mode, sms):
    cfg = CASES[name]
    M = cfg["neurons_per_module"]
    N = cfg["grid_w"] * cfg["grid_h"] * M
    Q = (N + 3) // 4
    bq, ptr, runs = snn.plan_pull_bands(cfg, sms, band_mode)
    # the bands tile the real quads in order
    assert bq[0] == 0 and bq[-1] == Q and np.all(np.diff(bq.astype(np.int64)) >= 0)
    sizes = np.diff(bq.astype(np.int64))
    if band_mode == 1:
        assert sizes.max() <= -(-Q // sms)
    else:
        for x in bq[1:-1]:
            assert x == Q or (int(x) * 4) % M == 0, x  # a module boundary on a quad boundary
        u = 4 // np.gcd(M, 4)
        units = -(-(N // M) // u)
        assert sizes.max() * 4 <= -(-units // sms) * u * M + 3
    assert ptr[0] == 0 and ptr[-1] == len(runs) and np.all(np.diff(ptr.astype(np.int64)) >= 0)
    if sms > Q:  # more SMs than quads: the trailing bands are empty
        assert np.count_nonzero(sizes) <= Q
    step = max(1, sms // 12)  # the brute force over every source is slow in Python: a spread of bands
    for b in list(range(0, sms, step)) + [sms - 1]:
        n0, n1 = int(bq[b]) * 4, min(int(bq[b + 1]) * 4, N)
        got = [(int(s), int(j) & 0xFFFF, int(j) >> 16) for s, j in runs[ptr[b]:ptr[b + 1]]]
        if n1 <= n0:
            assert got == []
            continue
        assert sorted(got) == _brute_runs(cfg, n0, n1), (name, b)


def test_module_aligned_bands_of_the_benchmark_network(snn):
    """24x24 x 1,250 neurons on 152 SMs: bands of 2 or 4 modules (boundaries
    every second module, where a module boundary falls on a quad), all SMs
    busy, no band reading a module it does not own."""
    cfg = CASES["gauss_24x24_M1250"]
    bq, ptr, runs = snn.plan_pull_bands(cfg, 152, 2)
    mods = np.diff(bq.astype(np.int64)) * 4 / 1250
    assert set(np.round(mods).astype(int)) == {2, 4} and np.all(mods > 0)
    assert sorted(np.round(mods).astype(int).tolist()).count(2) == 16  # 288 units of 2 modules over 152 SMs


def test_plan_argument_errors(snn):
    cfg = CASES["spec_4x4_M1000"]
    with pytest.raises(snn.SnnError, match="band_mode"):
        snn.plan_pull_bands(cfg, 152, 0)
    with pytest.raises(snn.SnnError, match="sms"):
        snn.plan_pull_bands(cfg, 0, 1)
