"""The C-ABI library builds, loads and exports every symbol the headers declare
(no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(crp_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libcrp():
    import paper_1210_0461_gb300 as pkg
    pkg.build()
    from paper_1210_0461_gb300 import crp
    return crp.lib()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for core in ("crp_plan_create", "crp_outer_accumulate", "crp_topk", "crp_sync",
                 "crp_partition_of", "crp_export_partitions", "crp_stats", "crp_plan_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(libcrp):
    missing = [n for n in declared_functions() if not hasattr(libcrp, n)]
    assert not missing, missing
    from paper_1210_0461_gb300 import crp
    out = subprocess.run(["nm", "-D", "--defined-only", crp.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\b(crp_[a-z0-9_]+)\b", out))
    assert set(declared_functions()) <= exported


def test_binding_signatures_cover_declared_symbols(libcrp):
    from paper_1210_0461_gb300 import crp
    assert set(declared_functions()) <= set(crp.exported_symbols())


def test_version_and_struct_sizes(libcrp):
    from paper_1210_0461_gb300 import crp
    assert libcrp.crp_version().startswith(b"crp ")
    assert ctypes.sizeof(crp.crp_sparse) == 48
    assert ctypes.sizeof(crp.crp_plan_desc) == 96
    assert ctypes.sizeof(crp.crp_stats_t) == 80


def test_sm103a_only_build_flags():
    from paper_1210_0461_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_no_cpu_fallback_in_binding():
    # The binding must not reach the oracle or any CPU implementation.
    src = open(os.path.join(ROOT, "paper_1210_0461_gb300", "crp.py")).read()
    assert "oracle" not in src.replace("no fallback", "")
    for f in glob.glob(os.path.join(ROOT, "paper_1210_0461_gb300", "*.py")):
        assert "import oracle" not in open(f).read() and "from oracle" not in open(f).read()
