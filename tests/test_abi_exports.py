"""The C-ABI library builds, loads without a GPU and exports every function include/rchfsi.h
declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_2503_22652_gb300 import build as B
from paper_2503_22652_gb300 import _lib

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rchfsi.h")


def declared_functions():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rchfsi_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("rchfsi_create", "rchfsi_destroy", "rchfsi_set_operator", "rchfsi_filter", "rchfsi_solve",
                 "rchfsi_submit", "rchfsi_poll", "rchfsi_strerror"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_strerror_without_gpu():
    lib = _lib.load()
    assert lib.rchfsi_strerror(0) == b"ok"
    assert b"invalid" in lib.rchfsi_strerror(-1)
    p = _lib.rchfsi_params()
    assert lib.rchfsi_params_default(ctypes.byref(p)) == 0
    assert p.degree == 20 and p.tol == 1e-8 and p.lanczos_steps == 10
