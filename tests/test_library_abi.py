"""The C-ABI library builds, loads and exports every symbol include/*.h declares
(no compute calls: these run without a GPU)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(sinn_[a-z_0-9]+)\s*\(",
                                src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2301_10622_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    need = {"sinn_create", "sinn_create_ex", "sinn_destroy", "sinn_insert", "sinn_delete",
            "sinn_search", "sinn_search_kp", "sinn_stats", "sinn_strerror"}
    assert need <= _declared()


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = _declared() - exported
    assert not missing, missing


def test_binding_loads_and_names_match(lib_path):
    from paper_2301_10622_gb300 import sinnamon
    lib = sinnamon.load()
    assert set(sinnamon.EXPORTS) == _declared()
    for name in sinnamon.EXPORTS:
        assert hasattr(lib, name)
    assert sinnamon.sinn_strerror(0) == "ok"
    assert sinnamon.sinn_strerror(2) == "id not live"


def test_library_targets_sm103a(lib_path):
    from paper_2301_10622_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_bounds_checked_build_exports_the_same_boundary(lib_path):
    """The -DSINN_BOUNDS_CHECK build (libsinnamon_bc.so) is the same library
    with index checks compiled in: it builds for sm_103a and exports the same
    declared symbols."""
    from paper_2301_10622_gb300 import build
    bc = build.build(bounds_check=True)
    assert bc != lib_path and os.path.basename(bc) == "libsinnamon_bc.so"

    def exported(path):
        out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                             text=True, check=True).stdout
        return {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert _declared() <= exported(bc)
    assert {s for s in exported(bc) if s.startswith("sinn_")} == \
        {s for s in exported(lib_path) if s.startswith("sinn_")}


def test_status_codes_have_names():
    from paper_2301_10622_gb300 import sinnamon
    sinnamon.load()
    names = [sinnamon.sinn_strerror(c) for c in range(sinnamon.SINN_EIO + 1)]
    assert len(set(names)) == len(names) and "unknown error" not in names
    assert sinnamon.sinn_strerror(99) == "unknown error"
