"""The C-ABI library builds, loads and exports every declared symbol; host-side
argument checks work without a GPU (no compute call is made here)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1608_07411_gb300 import build_lib, octfuse

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return octfuse.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "octfuse.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ofu_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ofu_create_octree", "ofu_integrate_frames", "ofu_iterate", "ofu_restructure",
              "ofu_energy", "ofu_export_leaves", "ofu_destroy", "ofu_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build_lib.OUT], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (ofu_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        getattr(lib, n)
    # the binding wraps each one under the same name
    assert set(_declared()) <= set(octfuse.exported_symbols())
    for n in _declared():
        assert callable(getattr(octfuse, n))


def test_params_layout_matches_header(lib):
    p = octfuse.ofu_default_params()
    assert p.max_depth == 6 and p.extent == 1.0 and p.spread_tau == 0.1
    assert abs(p.delta - 4 / 64) < 1e-15 and abs(p.eta - 8 / 64) < 1e-15
    assert p.lambda_ == 0.5 and p.gamma == 1e-3 and p.tau_split == 0.95 and p.tau_join == 0.99
    assert list(p.origin) == [-0.5, -0.5, -0.5] and p.max_leaves == 0 and p.data_term == 0
    assert ctypes.sizeof(octfuse.Params) == 3 * 8 + 8 + 4 + 4 + 7 * 8 + 8 + 4 + 4


@pytest.mark.parametrize("field,value,msg", [
    ("max_depth", 0, "max_depth"), ("max_depth", 16, "max_depth"), ("extent", -1.0, "extent"),
    ("delta", 0.0, "delta"), ("gamma", 0.0, "gamma"), ("lambda_", float("nan"), "lambda"),
    ("tau_join", 0.5, "tau_join"), ("sample_fp16", 2, "sample_fp16"), ("max_leaves", -5, "max_leaves"),
    ("data_term", 2, "data_term"), ("reserved", 1, "reserved"),
])
def test_invalid_params_rejected_on_host(lib, field, value, msg):
    p = octfuse.ofu_default_params()
    setattr(p, field, value)
    with pytest.raises(octfuse.OfuError) as e:
        octfuse.ofu_create_octree(p)
    assert e.value.status == octfuse.OFU_EINVAL and msg in str(e.value)


def test_null_arguments(lib):
    assert lib.ofu_create_octree(None, None, None) == octfuse.OFU_EINVAL
    assert lib.ofu_iterate(None, 1) == octfuse.OFU_EINVAL
    assert lib.ofu_energy(None, None, None, None) == octfuse.OFU_EINVAL
    lib.ofu_destroy(None)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(octfuse, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        octfuse.load(str(tmp_path / "nope.so"))


def test_allocator_callbacks_come_in_pairs(lib):
    p = octfuse.ofu_default_params()
    out = ctypes.c_void_p()
    alloc = octfuse.ALLOC_FN(lambda n, user: None)
    st = lib.ofu_create_octree_ex(ctypes.byref(p), None, alloc, octfuse.FREE_FN(), None,
                                  ctypes.byref(out))
    assert st == octfuse.OFU_EINVAL and out.value is None
    assert "both" in octfuse.ofu_last_error()
