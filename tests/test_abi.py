"""CPU checks of the boundary: the library builds, loads and exports every
symbol include/ptadd.h declares; host-side argument logic; the product
package never reaches the oracle.  No compute call needs a GPU here."""

import ast
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2005_02498_gb300")


def header_functions():
    txt = open(os.path.join(ROOT, "include", "ptadd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ptadd_[a-z0-9_]+)\s*\(", txt)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2005_02498_gb300 import build, ptadd
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = header_functions()
    assert len(declared) >= 16
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(ptadd.EXPORTS) == [n for n in declared if n in ptadd.EXPORTS]
    missing = [n for n in declared if n not in ptadd.EXPORTS]
    assert not missing, "binding does not wrap: %s" % missing


def test_version_and_error_string_without_gpu():
    from paper_2005_02498_gb300 import ptadd
    lib = ptadd.load()
    assert lib.ptadd_version() == 2
    assert isinstance(lib.ptadd_last_error(), bytes)


def test_create_rejects_bad_material_before_touching_a_device():
    from paper_2005_02498_gb300 import ptadd
    lib = ptadd.load()
    h = ctypes.c_void_p()
    bad = ptadd.Material(-1.0, 0.3, 2.5e-10, 2.5e-10, 1e-4)
    assert lib.ptadd_create(ctypes.byref(h), ctypes.byref(bad), 0, 0) == 1  # PTADD_ERR_ARG
    assert b"material" in lib.ptadd_last_error()
    good = ptadd.Material(48e9, 0.34, 2.556e-10, 2.556e-10, 1e-4)
    assert lib.ptadd_create(ctypes.byref(h), ctypes.byref(good), 7, 0) == 1  # unknown precision
    assert lib.ptadd_create(None, ctypes.byref(good), 0, 0) == 1


def test_null_context_calls_fail_cleanly():
    from paper_2005_02498_gb300 import ptadd
    lib = ptadd.load()
    assert lib.ptadd_set_applied_stress(None, None) == 1
    assert lib.ptadd_get_info(None, None) == 1
    lib.ptadd_destroy(None)


def _imports(path):
    tree = ast.parse(open(path).read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            names.add(node.module or "")
    return names


def test_product_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            p = os.path.join(dirpath, f)
            if f.endswith(".py"):
                assert not any(n == "oracle" or n.startswith("oracle.") for n in _imports(p)), p
            if f.endswith((".cu", ".cuh", ".h", ".py")):
                txt = open(p).read()
                assert "ptadd_oracle" not in txt and "liboracle" not in txt, p


def test_oracle_builds_and_reports_threads():
    import oracle
    assert oracle.num_threads() >= 1


def test_source_hash_follows_the_sources(tmp_path, monkeypatch):
    """The autotuner's cache key part that names the build: the same for the
    same sources, different when a CUDA source or the public header changes."""
    import shutil
    from paper_2005_02498_gb300 import build as B
    shutil.copytree(B.CSRC, tmp_path / "pkg" / "csrc")
    shutil.copytree(os.path.join(B.ROOT, "include"), tmp_path / "include")
    monkeypatch.setattr(B, "CSRC", str(tmp_path / "pkg" / "csrc"))
    monkeypatch.setattr(B, "ROOT", str(tmp_path))
    h0 = B.source_hash()
    assert h0 == B.source_hash() and len(h0) == 16 and int(h0, 16) >= 0
    for rel in ("pkg/csrc/pair_tile.cuh", "pkg/csrc/batch.cu", "include/ptadd.h"):
        f = tmp_path / rel
        text = f.read_text()
        f.write_text(text + "\n// changed\n")
        assert B.source_hash() != h0, rel
        f.write_text(text)
        assert B.source_hash() == h0
    (tmp_path / "pkg" / "csrc" / "notes.txt").write_text("not a source")
    assert B.source_hash() == h0
