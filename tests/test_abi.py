"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/gbmc.h declares; argument errors are reported before any device work.
No compute call is made here (this suite runs without a GPU)."""
import ctypes
import re

import pytest

from paper_1709_04394_gb300 import build as gbuild
from paper_1709_04394_gb300 import gbmc


def declared_functions():
    src = open(gbmc.HEADER_PATH).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return gbmc.load()


def test_header_declares_the_boundary_entry_points():
    names = declared_functions()
    for n in ("lattice_init", "metropolis_sweeps", "observables", "pa_step", "pa_run", "pa_create",
              "gbmc_create", "gbmc_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    for n in declared_functions():
        assert hasattr(gbmc, n), n


def test_argument_errors_before_device_work(lib):
    out = ctypes.c_void_p()
    assert lib.gbmc_create(None, 0, None) == gbmc.GBMC_ERR_ARG
    assert lib.lattice_init(None, None, None, 0, ctypes.byref(out)) == gbmc.GBMC_ERR_ARG
    assert b"NULL" in lib.gbmc_last_error()
    assert lib.metropolis_sweeps(None, None, 0.4, 1, None, None) == gbmc.GBMC_ERR_ARG
    assert lib.pa_run(None, None, None, 0, None) == gbmc.GBMC_ERR_ARG
    assert lib.lattice_free(None) == gbmc.GBMC_OK
    assert lib.gbmc_version() >= 100


def test_no_cpu_fallback_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(gbmc, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gbmc, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        gbmc.load()
