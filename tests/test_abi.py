"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/pibm.h declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from _util import ROOT, build_library


def _declared():
    src = open(os.path.join(ROOT, "include", "pibm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pibm_[a-z_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = _declared()
    for required in ("pibm_create", "pibm_destroy", "pibm_step", "pibm_set_particles", "pibm_set_markers",
                     "pibm_read_field", "pibm_read_particles", "pibm_read_particle_forces", "pibm_nusselt",
                     "pibm_read_contacts", "pibm_read_cells"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = build_library()
    assert os.path.exists(lib)
    L = ctypes.CDLL(lib)
    for name in _declared():
        assert hasattr(L, name), name
    nm = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(pibm_[a-z_]+)\b", nm))
    assert set(_declared()) <= exported


def test_binding_signatures_cover_header():
    from paper_1502_01159_gb300 import _native
    assert set(_native.SIGNATURES) == set(_declared())


def test_status_strings_without_gpu():
    from paper_1502_01159_gb300 import _native
    L = _native.load()
    assert L.pibm_status_string(0) == b"ok"
    assert L.pibm_status_string(5) == b"non-finite values"


def test_create_rejects_bad_description_before_touching_the_device():
    from paper_1502_01159_gb300 import _native
    L = _native.load()
    d = _native.pibm_desc()
    d.dim = 4  # invalid
    h = ctypes.c_void_p()
    st = L.pibm_create(ctypes.byref(d), None, None, ctypes.byref(h))
    assert st == _native.PIBM_ERR_ARG and not h.value
    buf = ctypes.create_string_buffer(128)
    L.pibm_last_error(None, buf, 128)
    assert b"lattice" in buf.value


def test_missing_library_fails_loudly(tmp_path):
    from paper_1502_01159_gb300 import _native
    with pytest.raises(RuntimeError, match="missing"):
        _native._lib_saved = _native._lib
        try:
            _native._lib = None
            _native.load(str(tmp_path / "libpibm.so"))
        finally:
            _native._lib = _native._lib_saved


def test_binding_constants_match_header_enums():
    # every PIBM_* enumerator of the header has the value the binding uses
    from paper_1502_01159_gb300 import _native
    src = open(os.path.join(ROOT, "include", "pibm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    values = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            name, _, val = item.partition("=")
            name = name.strip()
            nxt = int(val.strip(), 0) if val.strip() else nxt
            values[name] = nxt
            nxt += 1
    tunes = {k: v for k, v in values.items() if k.startswith("PIBM_TUNE_")}
    assert "PIBM_TUNE_LATTICE_PAIRS" in tunes
    for name, v in tunes.items():
        assert getattr(_native, name[len("PIBM_"):]) == v, name
    for name in ("PIBM_STORE_F32", "PIBM_STORE_F64", "PIBM_STORE_F16", "PIBM_STORE_BF16", "PIBM_HERTZ_MD_HIST"):
        if name in values:
            assert getattr(_native, name[len("PIBM_"):]) == values[name], name
