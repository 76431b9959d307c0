"""The C-ABI library builds, loads and exports what include/ehdlb.h declares.

Runs without a GPU: only entry points that touch no device are called.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2501_04920_gb300 import ehdlb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ehdlb.h")
GOLDEN = os.path.join(ROOT, "tests", "golden", "printed_values.txt")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ehdlb_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    L = ehdlb.lib()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name


def test_params_struct_matches_the_header_layout():
    # field names of ehdlb_params in declaration order, parsed from the header
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct ehdlb_params \{(.*?)\} ehdlb_params;", text, re.S).group(1)
    hdr = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, rest = decl.split(None, 1)
        hdr += [v.strip() for v in rest.split(",")]
    assert hdr == [n for n, _ in ehdlb._PARAM_FIELDS]
    p = ehdlb.ehdlb_params_default()
    assert p.size == C.sizeof(ehdlb.ehdlb_params)


def test_params_default_is_the_64x64_droplet_case():
    from paper_2501_04920_gb300 import workloads
    p = ehdlb.params_dict(ehdlb.ehdlb_params_default())
    w = workloads.droplet64()
    for k, v in w.items():
        assert p[k] == pytest.approx(v, rel=1e-15, abs=0), k


def test_params_from_physical_reproduces_printed_W0_and_beta():
    ny = 256
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        kv = dict(p.split("=") for p in parts[1:] if "=" in p)
        val = float([p for p in parts[1:] if "=" not in p][0])
        d, dpsi = float(kv["d_mm"]), float(kv.get("dpsi_kV", 1.0))
        p = ehdlb.ehdlb_params_from_physical(128, ny, d, dpsi, 0.5, 5.0)
        if parts[0] == "W0":
            assert p.Kq * ny * ny / dpsi == pytest.approx(val, rel=2e-5)
        else:
            assert np.sqrt(p.onsager_cb**2 * p.Kq * ny) == pytest.approx(val, rel=2e-4)


def test_null_and_bad_arguments_are_rejected_without_a_device():
    L = ehdlb.lib()
    assert L.ehdlb_step(None, 1, None) == ehdlb.EINVAL
    assert L.ehdlb_set_params(None, None) == ehdlb.EINVAL
    assert L.ehdlb_get_fields(None, 1, None, 0) == ehdlb.EINVAL
    assert L.ehdlb_params_default(None) == ehdlb.EINVAL
    assert L.ehdlb_set_reporting(None, 1, 0) == ehdlb.EINVAL
    h = C.c_void_p()
    assert L.ehdlb_create(C.byref(h), 3, 64, ehdlb.FP32, None) == ehdlb.EINVAL
    assert L.ehdlb_create(C.byref(h), 64, 64, 7, None) == ehdlb.EINVAL
    assert not h.value
    L.ehdlb_destroy(None)
    assert ehdlb.ehdlb_version() == 5


def test_batch_entry_points_reject_null_without_a_device():
    L = ehdlb.lib()
    h = C.c_void_p()
    assert L.ehdlb_batch_create(None, ehdlb.FP32, 1 << 20, 20, None) == ehdlb.EINVAL
    assert L.ehdlb_batch_create(C.byref(h), ehdlb.FP64, 1 << 20, 20, None) == ehdlb.EINVAL
    assert L.ehdlb_batch_create(C.byref(h), ehdlb.FP32, 1 << 20, 0, None) == ehdlb.EINVAL
    assert L.ehdlb_batch_step(None, 1, None) == ehdlb.EINVAL
    assert L.ehdlb_batch_remove(None, 0) == ehdlb.EINVAL
    assert L.ehdlb_batch_info(None, None, None, None) == ehdlb.EINVAL
    L.ehdlb_batch_destroy(None)


def test_batch_footprint_grows_with_the_lattice_and_halves_with_fp16_storage():
    f = ehdlb.ehdlb_batch_footprint
    a, b = f(ehdlb.FP32, 128, 128), f(ehdlb.FP32, 256, 256)
    assert 3.5 * a < b < 4.5 * a
    # per node: about 348 B in FP32 (two time levels of 27 populations,
    # g, auxiliary planes, snapshot, staging)
    assert 300 * 256 * 256 < b < 420 * 256 * 256
    assert f(ehdlb.FP16S, 256, 256) < 0.8 * b

