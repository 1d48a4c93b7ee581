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
    assert ctypes.sizeof(crp.crp_plan_desc) == 104
    assert ctypes.sizeof(crp.crp_stats_t) == 88


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets the C
    compiler gives the header's structs."""
    import shutil
    import subprocess
    from paper_1210_0461_gb300 import crp
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    checks = []
    for cname, ct in (("crp_sparse", crp.crp_sparse), ("crp_plan_desc", crp.crp_plan_desc),
                      ("crp_stats_t", crp.crp_stats_t)):
        checks.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in ct._fields_:
            checks.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "crp.h"\nint main(void){\n'
                   + "\n".join(checks) + "\nreturn 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for cname, ct in (("crp_sparse", crp.crp_sparse), ("crp_plan_desc", crp.crp_plan_desc),
                      ("crp_stats_t", crp.crp_stats_t)):
        assert int(got[cname]) == ctypes.sizeof(ct), cname
        for f, _ in ct._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(ct, f).offset, (cname, f)


def test_sm103a_only_build_flags():
    from paper_1210_0461_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_no_cpu_fallback_in_binding():
    # The binding must not reach the oracle or any CPU implementation.
    src = open(os.path.join(ROOT, "paper_1210_0461_gb300", "crp.py")).read()
    assert "oracle" not in src.replace("no fallback", "")
    for f in glob.glob(os.path.join(ROOT, "paper_1210_0461_gb300", "*.py")):
        assert "import oracle" not in open(f).read() and "from oracle" not in open(f).read()
