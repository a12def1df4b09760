"""The C-ABI library loads and exports every entry point include/pasfm.h declares (CPU).

Only host-side calls are made here (argument validation and workspace sizing
return before any CUDA work), so the test runs without a GPU.
"""
import ctypes
import os
import re

import pytest
import torch

from paper_2604_09643_b300 import binding, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pasfm_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_the_four_hot_path_calls():
    names = declared_symbols()
    for n in ("pasfm_forward", "pasfm_adjoint", "pasfm_pose_grad", "pasfm_step"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = binding.lib()
    for name in sorted(declared_symbols()):
        assert hasattr(L, name), name


def test_binding_covers_every_declared_symbol():
    assert declared_symbols() <= set(binding.symbols())


def test_abi_version():
    assert binding.lib().pasfm_abi_version() == 3


def _geom(**kw):
    g = synth.single_frame().geom
    g.update(kw)
    return binding.make_geom(g)


def test_workspace_size_is_host_only():
    n = ctypes.c_size_t(0)
    assert binding.lib().pasfm_workspace_size(ctypes.byref(_geom()), ctypes.byref(n)) == 0
    assert n.value > 0


@pytest.mark.parametrize("bad", [dict(dx=0.0), dict(fs_mhz=-1.0), dict(c_mm_per_us=0.0), dict(nx=-1),
                                 dict(n_samples=-5)])
def test_invalid_geometry_is_rejected(bad):
    n = ctypes.c_size_t(0)
    rc = binding.lib().pasfm_workspace_size(ctypes.byref(_geom(**bad)), ctypes.byref(n))
    assert rc == -1
    assert binding.lib().pasfm_last_error()


def test_unsupported_sphere_radius_is_reported():
    n = ctypes.c_size_t(0)
    rc = binding.lib().pasfm_workspace_size(ctypes.byref(_geom(a0_mm=1.0)), ctypes.byref(n))
    assert rc == -6


def test_null_context_is_rejected_without_cuda():
    L = binding.lib()
    g = _geom()
    assert L.pasfm_forward(None, ctypes.byref(g), None, None, None, None, None) == -1
    assert L.pasfm_adjoint(None, ctypes.byref(g), None, None, None, None, None) == -1
    assert L.pasfm_pose_grad(None, ctypes.byref(g), None, None, None, None, None, None, None, None) == -1
    assert L.pasfm_step(None, ctypes.byref(g), None, None, None, None, None, None, None, None) == -1
    assert b"ctx" in L.pasfm_last_error()


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device error path")
def test_create_without_device_fails_cleanly():
    h = ctypes.c_void_p()
    rc = binding.lib().pasfm_create(ctypes.byref(h), 0)
    assert rc == -3 and not h.value


def test_binding_refuses_host_tensors():
    with pytest.raises(ValueError):
        binding._ptr(torch.zeros(4), torch.float32, "x")


def test_wait_limit_needs_a_context():
    assert binding.lib().pasfm_set_wait_limit(None, 0) == -1
