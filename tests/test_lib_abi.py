"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/c2f.h declares (no device work: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

import paper_1905_09317_gb300 as c2f


def _declared():
    with open(os.path.join(ROOT, "include", "c2f.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"C2F_API\s+[\w\s\*]*?\b(c2f_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    c2f.build()
    return c2f.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("c2f_load_landscape", "c2f_set_weather", "c2f_simulate", "c2f_burn_prob"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", c2f.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(c2f_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert isinstance(getattr(lib, n), ctypes._CFuncPtr)
    # the binding declares exactly the header's entry points
    assert sorted(c2f.exported_symbols()) == _declared()


def test_defaults_and_no_device_path(lib):
    p = c2f.default_params()
    assert p.n_replicas == 1 and p.minutes_per_step == 1 and p.m1_pc == 50.0
    assert p.o1_curing_pct == 60.0 and p.outputs == (c2f.OUT_SCARS | c2f.OUT_COUNTERS)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        h = ctypes.c_void_p()
        assert lib.c2f_create(ctypes.byref(h), 0) == c2f.C2F_EINVAL
        with pytest.raises(c2f.C2FError):
            c2f.Context(0)
    # NULL context arguments are rejected without touching a device
    assert lib.c2f_simulate(None, 1, None, None) == c2f.C2F_EINVAL
    assert lib.c2f_release(None, 1) == c2f.C2F_EINVAL


def test_hooks_are_checked_before_any_device_call(lib):
    h = ctypes.c_void_p()
    bad = c2f.AllocHooks()            # NULL alloc / free
    assert lib.c2f_create_with_hooks(ctypes.byref(h), 0, ctypes.byref(bad)) == c2f.C2F_EINVAL
    assert lib.c2f_create_with_hooks(None, 0, None) == c2f.C2F_EINVAL
    assert lib.c2f_get_scar_bits(None, 1, None) == c2f.C2F_EINVAL
    assert lib.c2f_get_scars_at_hour(None, 1, 0, None) == c2f.C2F_EINVAL
