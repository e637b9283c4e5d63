"""The C-ABI library builds, loads and exports every symbol include/swe_gb300.h declares (CPU only)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "swe_gb300.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set()
    for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", txt):
        name = m.group(1)
        if name.startswith(("swe_", "sht_", "propagate_", "parareal_", "mgrit_")) and not name.endswith("_t"):
            names.add(name)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2306_09497_gb300 import build, swe
    if not os.path.exists(build.lib_path()):
        try:
            build.build()
        except Exception as e:  # pragma: no cover - nvcc missing
            pytest.skip(f"cannot build: {e}")
    return swe.load()


def test_header_and_binding_agree():
    from paper_2306_09497_gb300 import swe
    assert _declared() == set(swe.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    from paper_2306_09497_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.lib_path()], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = _declared() - exported
    assert not missing, f"missing exports: {missing}"
    for name in _declared():
        getattr(lib, name)


def test_host_only_calls(lib):
    from paper_2306_09497_gb300 import swe
    assert lib.swe_version().decode().startswith("swe_gb300")
    assert swe.ncoef(31) == 528
    assert swe.ncoef(255) == 32896
