"""The C-ABI library builds, loads and exports every entry point include/tgv.h declares.

Runs without a GPU: no call here launches device work.
"""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "tgv.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^TGV_API\s+[\w\s\*]+?\b(tgv_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2107_14790_b300 import build
    build.build()
    from paper_2107_14790_b300 import tgv
    return tgv.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("tgv_create_domain", "tgv_accumulate_depthmap", "tgv_solve", "tgv_extract_field",
                     "tgv_extract_histograms", "tgv_prolong", "tgv_destroy_domain", "tgv_status_string",
                     "tgv_last_error", "tgv_energy"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    for name in declared_symbols():
        assert hasattr(built_lib, name), name
        assert isinstance(getattr(built_lib, name), ctypes._CFuncPtr)


def test_binding_covers_every_declared_symbol(built_lib):
    from paper_2107_14790_b300 import tgv
    names = declared_symbols()
    bound = set(n for n in dir(tgv) if n.startswith("tgv_"))
    missing = [n for n in names if n not in bound and n not in ("tgv_default_params", "tgv_status_string",
                                                                "tgv_last_error")]
    assert not missing, missing


def test_host_only_entry_points(built_lib):
    from paper_2107_14790_b300 import tgv
    p = tgv.make_params(nbins=10, storage="bf16")
    assert p.nbins == 10 and p.storage == 1 and abs(p.tau - 0.2) < 1e-7 and abs(p.alpha0 - 2.0) < 1e-7
    assert built_lib.tgv_status_string(0) == b"ok"
    assert built_lib.tgv_status_string(3) == b"budget exceeded"
    assert built_lib.tgv_create_domain(None, 0, None, None, None) == 1  # null output pointer: invalid argument
    assert built_lib.tgv_level_voxels(None, 0) == 0
    assert built_lib.tgv_domain_bytes(None) == 0


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2107_14790_b300 import tgv
    monkeypatch.setattr(tgv, "_lib", None)
    monkeypatch.setattr(tgv, "_LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        tgv.lib()
