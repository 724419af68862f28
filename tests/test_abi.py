"""The C-ABI library builds for sm_103a, loads and exports every entry point
declared in include/matvis.h (no GPU needed: no compute call is made)."""
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "matvis.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mv_[a-z_]+)\s*\(", src)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not available")
def test_library_builds_loads_and_exports_header():
    from paper_2312_09763_gb300 import _build, binding
    path = _build.build()
    lib = binding.load_library(path)
    names = declared_entry_points()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing
    assert set(binding.EXPORTS) == set(names)


def test_product_has_no_cpu_fallback(tmp_path):
    from paper_2312_09763_gb300 import binding
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(ImportError):
            binding.load_library(str(tmp_path / "missing.so"))
    finally:
        binding._lib = saved


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2312_09763_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "matvis_oracle" not in txt, f
