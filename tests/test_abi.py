"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function include/snn.h declares; snn_config has the same layout
in C and in the binding; descriptions are validated before any CUDA call."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_1803_08833_gb300 import snn
from paper_1803_08833_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "snn.h")


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1803_08833_gb300 import _build
    _build.build()
    return snn.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SNN_API\s+[\w\s\*]+?\b(snn_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", snn.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(snn_\w+)", out))
    assert set(names) <= exported, set(names) - exported
    for n in names:
        assert hasattr(lib, n)
    # nothing but the ABI is exported
    assert exported == set(names)


def test_config_layout_matches_c(tmp_path):
    fields = [f[0] for f in snn.SnnConfig._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "snn.h"', "int main(void) {",
             'printf("%zu\\n", sizeof(snn_config));']
    lines += ['printf("%%zu\\n", offsetof(snn_config, %s));' % f for f in fields]
    lines += ['printf("%zu\\n", sizeof(snn_stats));', "return 0; }"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert vals[0] == ctypes.sizeof(snn.SnnConfig)
    assert vals[1:-1] == [getattr(snn.SnnConfig, f).offset for f in fields]
    assert vals[-1] == ctypes.sizeof(snn.SnnStats)


def _build_status(lib, cfg):
    c = snn.config(cfg)
    h = ctypes.c_void_p()
    st = lib.snn_build_network(ctypes.byref(c), snn.ALLOC_FN(), snn.FREE_FN(), None, None, ctypes.byref(h))
    return st, lib.snn_last_error().decode(), h.value


@pytest.mark.parametrize("bad,needle", [
    ({"grid_w": 0}, "grid"),
    ({"neurons_per_module": 0}, "grid"),
    ({"K": 20000}, "K must"),
    ({"kernel": 2}, "kernel"),
    ({"sigma_um": 0.0}, "sigma"),
    ({"d_exc_lo": 0}, "delays"),
    ({"d_exc_hi": 300}, "delays"),
    ({"d_inh": 0}, "delays"),
    ({"fx_shift": 30}, "fx_shift"),
    ({"weight_dtype": 7}, "weight_dtype"),
    ({"tau_m_ms": 0.0}, "tau"),
    ({"exc_fraction": 1.5}, "exc_fraction"),
    ({"w_exc_hi": float("inf")}, "non-finite"),
    ({"ext_rate_hz": -1.0}, "ext_rate"),
    ({"grid_w": 200, "grid_h": 200, "neurons_per_module": 1000}, "too many neurons"),
])
def test_invalid_descriptions_are_rejected(lib, bad, needle):
    cfg = W.small()
    cfg.update(bad)
    st, msg, h = _build_status(lib, cfg)
    assert st == snn.SNN_EINVAL and h is None
    assert needle in msg


def test_null_arguments(lib):
    assert lib.snn_step(None, 1, None) == snn.SNN_EINVAL
    assert lib.snn_clear_raster(None, None) == snn.SNN_EINVAL
    assert lib.snn_set_schedule(None, 0, 0) == snn.SNN_EINVAL
    c = snn.config(W.small())
    assert lib.snn_build_network(ctypes.byref(c), snn.ALLOC_FN(), snn.FREE_FN(), None, None, None) == snn.SNN_EINVAL
    lib.snn_destroy(None)


def test_allocator_hooks_must_come_in_pairs(lib):
    c = snn.config(W.small())
    h = ctypes.c_void_p()
    alloc = snn.ALLOC_FN(lambda n, ctx: None)
    st = lib.snn_build_network(ctypes.byref(c), alloc, snn.FREE_FN(), None, None, ctypes.byref(h))
    assert st == snn.SNN_EINVAL and "both" in lib.snn_last_error().decode()


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(snn, "_lib", None)
    monkeypatch.setattr(snn, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="libsnn.so not found"):
        snn.load()


def test_memory_estimate_tracks_the_table(lib):
    small = snn.estimate_bytes(W.gauss_4x4_k1000())
    big = snn.estimate_bytes(W.gauss_24x24_k1125())
    bf = snn.estimate_bytes(W.exp_24x24_k2250(weight_dtype="bf16"))
    f32 = snn.estimate_bytes(W.exp_24x24_k2250(weight_dtype="f32"))
    assert 128e6 < small < 400e6            # 16 M synapses x 8 B + state
    assert 6.5e9 < big < 7.0e9              # 810 M synapses x 8 B + ring
    assert bf < f32 and abs((f32 - bf) - 720000 * 2256 * 2) < 1e6
    # the pairwise rule: the longest-row bound sets the stride (Table I: ~1.25 k per neuron, 0.9 G in all)
    pw = snn.estimate_bytes(W.pairwise(grid=24))
    assert 0.9e9 * 8 < pw < 720000 * 1700 * 8
