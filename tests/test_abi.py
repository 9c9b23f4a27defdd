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
