"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and exports every
entry point the headers in include/ declare; the bindings name the same set; the product
path and the oracle share no code."""
import ctypes
import glob
import os
import re
import shutil
import subprocess

import pytest

from paper_1603_04334_gb300 import build as pkg_build
from paper_1603_04334_gb300 import batching, serve, sparc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def header_symbols(paths=HEADERS):
    syms = set()
    for path in paths:
        txt = open(path).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        syms |= set(re.findall(r"\b(sparc_[A-Za-z0-9_]+)\s*\(", txt))
    return sorted(syms)


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    return pkg_build.build()


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    syms = header_symbols()
    assert len(syms) >= 11
    for s in syms:
        assert hasattr(L, s), f"{s} declared in include/ but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (sparc_[A-Za-z0-9_]+)$", out, flags=re.M))
    assert set(syms) <= exported
    # nothing exported under sparc_ that the header does not declare
    assert exported <= set(syms), exported - set(syms)


def test_binding_names_match_header():
    assert sorted(sparc.EXPORTS + serve.EXPORTS + batching.EXPORTS) == header_symbols()


def test_library_is_built_for_sm103a(lib_path):
    cuobj = shutil.which("cuobjdump") or "/usr/local/cuda/bin/cuobjdump"
    if not os.path.exists(cuobj):
        pytest.skip("cuobjdump not available")
    # list the embedded ELF architectures only (no disassembly)
    out = subprocess.run([cuobj, "--list-elf", lib_path], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_product_and_oracle_share_no_code():
    pkg = os.path.join(ROOT, "paper_1603_04334_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "_lib" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, flags=re.M), f
                assert "sparc_oracle" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "libsparc_gb300" not in txt and "paper_1603_04334_gb300.sparc" not in txt, f
            assert "csrc" not in txt, f


def test_load_fails_loudly_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(pkg_build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(sparc, "_lib", None)
    with pytest.raises(RuntimeError):
        sparc.load(build_if_missing=False)
