"""snn_build_cdf_static: target-module tables built with no device allocation
by the library (for callers whose device memory belongs to a pool, or that
cannot afford cudaMalloc/cudaFree's device synchronisation).  Its output must
equal the tables the ordinary entry point, snn_build_network, builds -- on two
calls in a row, since every call reuses the same fixed scratch."""
import ctypes

import numpy as np
import pytest

from paper_1803_08833_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    from paper_1803_08833_gb300 import _build
    from paper_1803_08833_gb300 import snn
    _build.build()
    snn.load()
    return snn, torch


def _static_tables(snn, torch, cfg):
    L = snn.load()
    c = snn.config(cfg)
    mo = ctypes.c_uint32()
    snn.check(L.snn_build_cdf_static(ctypes.byref(c), None, None, None, ctypes.byref(mo), None))
    nm = cfg["grid_w"] * cfg["grid_h"]
    # caller-owned device buffers, filled with junk: every valid entry must be written
    T = torch.full((nm * mo.value,), -7, dtype=torch.int32, device="cuda")
    TM = torch.full((nm * mo.value,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((nm,), -7, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    snn.check(L.snn_build_cdf_static(ctypes.byref(c), ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(TM.data_ptr()),
                                     ctypes.c_void_p(cnt.data_ptr()), ctypes.byref(mo),
                                     ctypes.c_void_p(s.cuda_stream)))
    torch.cuda.synchronize()
    as_u32 = lambda x: x.cpu().numpy().view(np.uint32)
    return as_u32(T).reshape(nm, mo.value), as_u32(TM).reshape(nm, mo.value), as_u32(cnt)


def _network_tables(snn, cfg):
    with snn.Network(dict(cfg, neurons_per_module=2, K=8)) as net:
        return net.cdf()


def test_static_tables_equal_network_tables_on_consecutive_calls(env):
    snn, torch = env
    cases = [W.gauss_24x24_k1125(), W.exp_24x24_k2250(), dict(W.small(lateral="exp"), grid_w=13, grid_h=5)]
    for cfg in cases + cases[:1]:  # the last call reuses scratch left by a larger table
        T, TM, cnt = _static_tables(snn, torch, cfg)
        rT, rTM, rcnt = _network_tables(snn, cfg)
        assert T.shape == rT.shape
        assert np.array_equal(cnt, rcnt)
        for m in range(len(cnt)):
            n = cnt[m]
            assert np.array_equal(T[m, :n], rT[m, :n]), m
            assert np.array_equal(TM[m, :n], rTM[m, :n]), m


def test_static_rejects_tables_beyond_the_fixed_scratch(env):
    snn, torch = env
    cfg = dict(W.exp_24x24_k2250(), grid_w=48, grid_h=48)  # 2304 modules x 441 offsets > 524,288
    L = snn.load()
    c = snn.config(cfg)
    mo = ctypes.c_uint32()
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    st = L.snn_build_cdf_static(ctypes.byref(c), p, p, p, ctypes.byref(mo), None)
    assert st == snn.SNN_EINVAL
    assert "exceeds the fixed scratch" in L.snn_last_error().decode()
    assert mo.value == 441


def test_static_tables_under_stream_capture(env):
    """After a first call outside capture (the address lookup), a call inside a
    stream capture enqueues only kernels; replaying the graph writes the same
    tables as snn_build_network."""
    snn, torch = env
    cfg = W.exp_24x24_k2250()
    _static_tables(snn, torch, cfg)  # first call on this device: symbol lookup outside capture
    L = snn.load()
    c = snn.config(cfg)
    mo = ctypes.c_uint32()
    snn.check(L.snn_build_cdf_static(ctypes.byref(c), None, None, None, ctypes.byref(mo), None))
    nm = cfg["grid_w"] * cfg["grid_h"]
    T = torch.full((nm * mo.value,), -7, dtype=torch.int32, device="cuda")
    TM = torch.full((nm * mo.value,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((nm,), -7, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        st = L.snn_build_cdf_static(ctypes.byref(c), ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(TM.data_ptr()),
                                    ctypes.c_void_p(cnt.data_ptr()), ctypes.byref(mo), ctypes.c_void_p(s.cuda_stream))
        g.capture_end()
    snn.check(st)
    assert int(cnt[0].item()) == -7  # captured, not run
    g.replay()
    torch.cuda.synchronize()
    as_u32 = lambda x: x.cpu().numpy().view(np.uint32)
    T, TM, cnt = as_u32(T).reshape(nm, mo.value), as_u32(TM).reshape(nm, mo.value), as_u32(cnt)
    rT, rTM, rcnt = _network_tables(snn, cfg)
    assert np.array_equal(cnt, rcnt)
    for m in range(len(cnt)):
        n = cnt[m]
        assert np.array_equal(T[m, :n], rT[m, :n]), m
        assert np.array_equal(TM[m, :n], rTM[m, :n]), m
