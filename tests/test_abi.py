"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/fsgpu.h; the Python binding declares each of them.
No GPU is needed and no compute call is made."""

import ctypes
import os
import re

import pytest

from paper_2605_03123_gb300 import build, fsgpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fs_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def libpath():
    p = build.lib_path()
    if not os.path.exists(p):
        build.build()
    return p


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fs_apply_orbital_rotation", "fs_apply_diag_coulomb_evolution",
                     "fs_apply_num_op_sum_evolution", "fs_lucj_forward", "fs_lucj_vjp"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(libpath):
    assert declared_functions() <= set(fsgpu.SIGNATURES)
    fsgpu.load_library(libpath)


def test_build_targets_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
