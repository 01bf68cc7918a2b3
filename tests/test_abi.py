"""Host-side checks of the C ABI: the library exports every entry point declared in include/*.h,
and the Python binding carries the same names (no GPU needed; nothing is computed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ["lap_apply", "cheb_filter_spectrum", "rat_mass_solve", "gauge_force", "kinetic_force",
              "rmhmc_trajectory", "rmhmc_create", "rmhmc_destroy", "wilson_flow"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as ge
    so = ge.build_library()
    lib = ctypes.CDLL(so)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match():
    import paper_2112_04556_gb300 as rm
    for n in ["lap_apply", "cheb_filter_spectrum", "rat_mass_solve", "gauge_force", "kinetic_force",
              "rmhmc_trajectory", "lap_link_grad", "heatbath", "mass_fit", "wilson_flow"]:
        assert callable(getattr(rm, n))


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without librmhmc.so every entry point raises instead of computing elsewhere."""
    import paper_2112_04556_gb300 as rm
    monkeypatch.setattr(rm, "_SO", str(tmp_path / "missing.so"))
    monkeypatch.setattr(rm, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        rm.lib()
    with pytest.raises(RuntimeError):
        rm.window_coeffs([0.0, 1.0], 4)
