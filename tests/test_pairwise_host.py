"""The library's host-derived construction tables of the pairwise law and of
the efficacy / delay distributions against the oracle's independent
derivation (host code through the C ABI; no GPU work)."""
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


CASES = [
    W.pairwise(grid=24, lateral="gauss"),
    W.pairwise(grid=24, lateral="exp"),
    W.pairwise(grid=8, M=300, lateral="gauss", p_local=0.5, A_remote=0.2, p_min=1e-4),
    W.pairwise(grid=8, lateral="exp", spacing_um=400.0, lambda_um=240.0, p_local=1.0),
    W.pairwise(grid=6, M=50, w_exc_sd=0.3, w_inh_sd=0.05, delay_tau_ms=2.5, d_exc_lo=2, d_exc_hi=9),
]


@pytest.mark.parametrize("k", range(len(CASES)))
def test_tables_equal_the_oracle(snn, k):
    cfg = CASES[k]
    t = snn.construction_tables(cfg)
    dx, dy, _, thr = oracle.pair_stencil(cfg)
    assert np.array_equal(t["pair_dx"], dx) and np.array_equal(t["pair_dy"], dy)
    assert np.array_equal(t["pair_thr"], thr)
    we, _ = oracle.weight_table(cfg, True)
    wi, _ = oracle.weight_table(cfg, False)
    assert np.array_equal(t["wtab_exc"].view(np.uint32), we.view(np.uint32))
    assert np.array_equal(t["wtab_inh"].view(np.uint32), wi.view(np.uint32))
    assert np.array_equal(t["dthr"], oracle.delay_table(cfg))


def test_fixed_rule_has_no_stencil_and_uniform_laws_no_tables(snn):
    t = snn.construction_tables(W.small())
    assert len(t["pair_dx"]) == 0 and len(t["dthr"]) == 0 and not t["wtab_exc"].any()


@pytest.mark.parametrize("bad", [
    {"p_local": 1.5}, {"A_remote": -0.1}, {"p_min": 0.0}, {"conn_rule": 2}, {"weight_dist": 3},
    {"delay_dist": "exp", "delay_tau_ms": 0.0}, {"table_layout": "grouped"}, {"neurons_per_module": 70000},
])
def test_invalid_pairwise_descriptions(snn, bad):
    cfg = dict(W.pairwise(grid=4, M=100), **bad)
    with pytest.raises(snn.SnnError):
        snn.construction_tables(cfg)
