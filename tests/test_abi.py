"""The C-ABI library builds, loads and exports every entry point include/sgw.h declares
(no compute calls: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

import paper_1812_03717_gb300 as P
from paper_1812_03717_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "sgw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgw_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    if not os.path.exists(B.LIB):
        B.build()
    return B.LIB


def test_header_declares_the_binding_exports():
    assert _declared() == sorted(P.EXPORTS)


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    syms = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [s for s in _declared() if s not in syms]
    assert not missing, missing


def test_library_loads_through_binding(lib_path):
    lib = P.load()
    for name in P.EXPORTS:
        assert hasattr(lib, name)


def test_no_gpu_fails_loudly(lib_path):
    """Without a usable device the library returns an error instead of computing anything."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import instances as I
    inst = I.tiny_fcc()
    with pytest.raises(P.SgwError):
        P.System.from_instance(inst, inst.kpoints[0].kq_frac)
