"""The C ABI library builds, loads and exports every declared entry point
(no GPU needed: nothing here launches a kernel)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fem_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_0905_2203_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fem_[a-z0-9_]+)", out))
    decl = declared_functions()
    assert len(decl) >= 20
    missing = [f for f in decl if f not in exported]
    assert not missing, missing


def test_binding_loads_and_binds_every_symbol():
    from paper_0905_2203_gb300 import binding
    for f in declared_functions():
        assert hasattr(binding, f), f
    assert "sm_103a" in binding.version()
    assert binding.fem_strerror(binding.FEM_ERR_DUP).decode().startswith("stream repeats")


def test_no_oracle_on_product_path():
    """The product package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_0905_2203_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "fem_oracle" not in txt, f
