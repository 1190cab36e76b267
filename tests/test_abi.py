"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads,
and exports every function that include/atkm.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(", src, flags=re.M):
            name = m.group(1)
            if name not in ("if", "defined"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2603_05194_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("atkm_plan_create", "atkm_plan_destroy", "dipolar_potential", "apply_H",
                     "pcg_ground_state", "apply_preconditioner", "atkm_energy_parts"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(libpath):
    from paper_2603_05194_gb300 import binding
    lib = binding.load_library(libpath)
    for n in declared_functions():
        assert getattr(lib, n).argtypes is not None, n
