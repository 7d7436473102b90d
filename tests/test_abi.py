"""The C-ABI library builds, loads and exports every function include/ipcsim.h declares (no GPU needed)."""
import os
import re
import subprocess

from paper_2609_25653_b300 import build, ipcsim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+(sim_[A-Za-z0-9_]+)\s*\(", src, re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    decl = declared_functions()
    assert len(decl) >= 13
    missing = decl - exported
    assert not missing, missing
    L = ipcsim.load()
    for name in decl:
        assert hasattr(L, name)
    assert set(ipcsim.SIGNATURES) <= decl


def test_binding_refuses_missing_library(monkeypatch):
    import pytest
    monkeypatch.setattr(ipcsim, "LIB_PATH", "/nonexistent/libipcsim.so")
    monkeypatch.setattr(ipcsim, "_lib", None)
    with pytest.raises(ImportError):
        ipcsim.load()
