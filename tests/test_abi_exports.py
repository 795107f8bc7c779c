"""The C-ABI library loads on any machine and exports every declared call."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fedfem.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fedfem_\w+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1909_05098_gb300.build import build
    build()
    from paper_1909_05098_gb300 import fedfem
    lib = fedfem.library()
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert fedfem.fedfem_version().startswith("fedfem-gb300")
