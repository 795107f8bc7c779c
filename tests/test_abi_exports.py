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


def test_library_exports_no_other_c_symbols():
    """Every unmangled (C-linkage) function the library defines is one the
    header declares: internal helpers keep internal or C++ linkage."""
    import shutil
    import subprocess
    import pytest
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    from paper_1909_05098_gb300.build import build
    path = build()
    out = subprocess.run([nm, "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    c_funcs = {f[2] for f in (line.split() for line in out.splitlines()) if len(f) == 3 and f[1] == "T"
               and not f[2].startswith("_")}
    extra = sorted(c_funcs - set(declared_functions()))
    assert not extra, extra
