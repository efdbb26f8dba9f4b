"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/ankh.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2212_08284_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ankh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ankh_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("ankh_create", "ankh_energy", "ankh_energy_forces", "ankh_destroy", "ankh_last_error"):
        assert s in syms


def test_library_builds_and_exports_all_symbols():
    path = build.build()
    lib = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(api.EXPORTED) <= set(declared_symbols())


def test_version_and_defaults_without_gpu():
    lib = api.load_library()
    assert lib.ankh_version() >= 100
    p = api.ankh_default_params()
    assert p.xi == pytest.approx(0.01)
    assert p.Lu == 0 and p.n_cells == 0 and p.max_order == 2   # orders and leaf count from the accuracy table
    assert p.flags & api.ANKH_INCLUDE_REC


def test_invalid_arguments_rejected_on_host():
    """Argument validation happens before any device call."""
    p = api.ankh_default_params()
    p.Lu = 11
    with pytest.raises(api.AnkhError) as e:
        api.ankh_create(20.0, 100, p)
    assert e.value.code == api.ANKH_EINVAL
    with pytest.raises(api.AnkhError) as e:
        api.ankh_create(-1.0, 100)
    assert e.value.code == api.ANKH_EINVAL
    p = api.ankh_default_params()
    p.n_cells = 2
    with pytest.raises(api.AnkhError) as e:
        api.ankh_create(20.0, 100, p)
    assert e.value.code == api.ANKH_EINVAL
    with pytest.raises(api.AnkhError) as e:
        api.ankh_create(20.0, 0)
    assert e.value.code == api.ANKH_EINVAL
