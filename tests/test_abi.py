"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/*.h declares; its compiled-in constants agree with the input module
and the oracle.  No compute call: these run without a GPU."""
import glob
import os
import re

import numpy as np

from paper_2407_10797_gb300 import build, fstat
from paper_2407_10797_gb300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"FS_API\s+[\w\s\*]*?\b(fs_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = fstat.load()
    names = declared_symbols()
    assert {"fs_plan_create", "fs_fstat_batch", "fs_plan_destroy", "fs_last_error"} <= names
    for n in sorted(names):
        assert hasattr(L, n), n


def test_library_is_built_for_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.LIB)


def test_constants_agree():
    c = fstat.constants()
    assert c[0] == S.MSUN_S and c[1] == S.YEAR_S and c[2] == S.AU_S and c[3] == 0.01
    src = open(os.path.join(ROOT, "oracle", "fstat_oracle.c")).read()
    assert f"#define OR_F0_ECC {c[3]}" in src


def test_headers_are_plain_c_and_cpp():
    """Every include/*.h compiles on its own as strict C99 and C11 (pedantic,
    warnings as errors) and as C++ through its extern "C" guards: the boundary
    carries only plain C types."""
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    if cc is None:
        import pytest
        pytest.skip("gcc not found")
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        src = f'#include "{os.path.basename(h)}"\nint fs_header_check(void) {{ return 0; }}\n'
        for lang, std in (("c", "-std=c99"), ("c", "-std=c11"), ("c++", "-std=c++17")):
            r = subprocess.run([cc, "-x", lang, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                                "-I", os.path.join(ROOT, "include"), "-"], input=src, capture_output=True,
                               text=True)
            assert r.returncode == 0, (h, lang, std, r.stderr)
