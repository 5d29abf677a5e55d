"""CPU checks of the C ABI library: it builds, loads without a GPU, exports
every entry point that include/vplbm.h declares, and validates descriptors
on the host before touching a device."""
import ctypes
import os
import re

import pytest

import paper_1905_05110_gb300 as vp
import workloads as wl
from paper_1905_05110_gb300 import build as vbuild

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "vplbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vplbm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    vbuild.build()
    return vp.load_library()


def test_header_declares_the_bound_entry_points():
    assert declared_functions() == sorted(vp.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(vbuild.LIB)
    for name in declared_functions():
        assert hasattr(raw, name), name


def test_version_and_error_strings(lib):
    assert "vplbm" in vp.vplbm_version()
    assert isinstance(vp.vplbm_last_error(), str)


def test_buffer_sizes_scale_with_precision(lib):
    p = wl.channel_fixed_disk()
    sizes = {prec: vp.vplbm_buffer_sizes_for(vp.lattice_desc(p, prec), vp.body_desc(p["body"]), 100)
             for prec in ("f64", "f32", "f16")}
    n_pad = ((256 * 128 + 127) // 128) * 128
    assert sizes["f64"].populations == 9 * n_pad * 8
    assert sizes["f32"].populations == 9 * n_pad * 4
    assert sizes["f16"].populations == 9 * n_pad * 2
    assert sizes["f32"].history == 100 * 16 * 8
    assert sizes["f32"].partials % 256 == 0 and sizes["f32"].partials >= 8 * 8


@pytest.mark.parametrize("mutate,status", [
    (lambda p: p.update(nx=2), 1),
    (lambda p: p["s"].__setitem__(7, 2.0), 1),
    (lambda p: p.update(eta=0.0), 1),
    (lambda p: p["bc"].__setitem__("east", {"kind": "periodic"}), 1),
    (lambda p: p["bc"].__setitem__("north", {"kind": "zerograd"}), 6),
])
def test_invalid_lattice_rejected_on_host(lib, mutate, status):
    p = wl.channel_fixed_disk()
    p["s"] = list(p["s"])
    mutate(p)
    with pytest.raises(vp.VplbmError) as ei:
        vp.vplbm_buffer_sizes_for(vp.lattice_desc(p, "f32"), vp.body_desc(p["body"]), 10)
    assert ei.value.status == status


def test_invalid_body_rejected_on_host(lib):
    p = wl.sedimenting_disk(nx=64, ny=64, diameter=8)
    b = dict(p["body"])
    b["mass"] = 0.0
    with pytest.raises(vp.VplbmError) as ei:
        vp.vplbm_buffer_sizes_for(vp.lattice_desc(p, "f32"), vp.body_desc(b), 10)
    assert ei.value.status == 1
    b = dict(p["body"])
    b["x"] = float("nan")
    with pytest.raises(vp.VplbmError):
        vp.vplbm_buffer_sizes_for(vp.lattice_desc(p, "f32"), vp.body_desc(b), 10)
    with pytest.raises(vp.VplbmError):
        vp.vplbm_buffer_sizes_for(vp.lattice_desc(p, "f32"), vp.body_desc(p["body"]), 0)
