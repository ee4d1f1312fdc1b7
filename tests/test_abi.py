"""The C ABI library loads and exports every symbol include/sv.h declares.

CPU only: the library is loaded (a CUDA driver is not needed for that) and
only entry points that reject their arguments on the host are called.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2605_15098_gb300 import build as B
from paper_2605_15098_gb300 import circuits as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def svlib():
    B.build()
    from paper_2605_15098_gb300 import sv
    return sv


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\**\s*(sv_[a-z_0-9]+)\s*\(",
                            text, flags=re.M)
    return sorted(set(names))


def test_header_declares_boundary():
    names = declared_functions()
    for required in ("sv_create", "sv_apply_circuit", "sv_probabilities", "sv_sample",
                     "sv_destroy", "sv_argmax"):
        assert required in names


def test_exports_every_declared_symbol(svlib):
    lib = svlib.lib()
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported"
    assert set(svlib.EXPORTS) <= set(declared_functions())


def test_version(svlib):
    assert "sm_103a" in svlib.sv_version()


def test_gate_record_layout(svlib):
    assert C.GATE_DTYPE.itemsize == 96
    assert ctypes.sizeof(svlib.sv_config) == 64


def test_host_validation_rejects_without_device(svlib):
    lib = svlib.lib()
    h = ctypes.c_void_p()
    assert lib.sv_create(0, 0, ctypes.byref(h)) == svlib.SV_ERR_ARG
    assert "outside" in svlib.sv_last_error()
    assert lib.sv_create(35, 0, ctypes.byref(h)) == svlib.SV_ERR_ARG
    assert lib.sv_create(5, 7, ctypes.byref(h)) == svlib.SV_ERR_ARG
    assert lib.sv_create(5, 0, None) == svlib.SV_ERR_ARG
    assert lib.sv_destroy(None) == svlib.SV_OK
    assert lib.sv_apply_circuit(None, None, 0, None) == svlib.SV_ERR_ARG
    assert lib.sv_create_on(5, 0, None, 0, None, ctypes.byref(h)) == svlib.SV_ERR_ARG
    g = C.gates([C.h(0)])
    assert lib.sv_apply_circuit(None, g.ctypes.data, 1, None) == svlib.SV_ERR_ARG
    # misaligned adopted buffer is refused before any CUDA call
    assert lib.sv_create_on(5, 0, ctypes.c_void_p(16), 1 << 20, None,
                            ctypes.byref(h)) == svlib.SV_ERR_ARG
    assert "aligned" in svlib.sv_last_error()


def test_batch_host_path_without_device(svlib):
    """sv_batch_create plans and packs every item on the host before any CUDA
    call; without a device it must stop with SV_ERR_CUDA, not crash."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("host-only check")
    work = C.qpe_batch(40, seed=5)
    with pytest.raises(svlib.SvError) as e:
        svlib.sv_batch_create([(n, g, m) for n, g, m, _ in work])
    assert e.value.code == svlib.SV_ERR_CUDA
    bad = [(5, C.gates([C.h(7)]), 1)]
    with pytest.raises(svlib.SvError) as e:
        svlib.sv_batch_create(bad)
    assert e.value.code == svlib.SV_ERR_ARG


def test_cost_features_host(svlib):
    """Feature vector layout of a launch record (host only)."""
    rec = {"kind": svlib.SV_KERNEL_TILE, "n": 28, "k": 13, "c": 5, "ngates": 15, "dtype": 0,
           "gate_kind": -2, "bytes": 4.0e9, "feat": (1 << 5) - 1 | (1 << 9) | (1 << 27),
           "stages": 3, "blocks": 0, "nins": 40, "nfactors": 7}
    f = svlib.sv_cost_features(rec)
    assert f.shape == (svlib.SV_COST_FEATURES,)
    assert list(f[:32]) == [float((rec["feat"] >> q) & 1) for q in range(32)]
    assert list(f[32:36]) == [0, 0, 0, 1]        # top qubit 27 >= k
    assert list(f[36:38]) == [0, 0]              # reads its tile; complex64
    assert list(f[38:43]) == [0, 0, 1, 0, 0]     # register-stage kernel
    assert abs(f[43] - np.log2(16) / 8) < 1e-6
    assert abs(f[47] - 5 / 16) < 1e-7 and abs(f[49] - 13 / 16) < 1e-7 and abs(f[51] - 8 / 16) < 1e-7
    rec.update(kind=svlib.SV_KERNEL_REMAP, gate_kind=-4, feat=(1 << 3) | (1 << 20))
    f = svlib.sv_cost_features(rec)
    assert list(f[38:43]) == [0, 0, 0, 0, 1] and list(f[32:36]) == [0, 0, 0, 1]
    rec.update(kind=svlib.SV_KERNEL_FUSED, gate_kind=-3, feat=0b111, dtype=1)
    f = svlib.sv_cost_features(rec)
    assert list(f[38:43]) == [0, 0, 0, 1, 0] and list(f[32:36]) == [1, 0, 0, 0]
    assert list(f[36:38]) == [0, 1]              # complex128
    rec.update(kind=svlib.SV_KERNEL_TILE, gate_kind=-2, dtype=0, generated=1)
    f = svlib.sv_cost_features(rec)
    assert list(f[36:38]) == [1, 0]              # generates its state
    assert svlib.cost_target({"ms": 2.0, "bytes": 4.0e9}) == pytest.approx(np.log(0.5))
