"""The oracle and the CUDA path share no code: the package (Python binding,
build step, CUDA sources) neither imports nor includes anything under
oracle/, the oracle neither imports the package nor includes its headers,
and the two scripts that may run the oracle outside the tests (bench.py's
CPU baseline and reference arm, the smoke check) import it only inside
those functions (the build step also compiles the C oracle)."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2407_10797_gb300")


def _imports(tree):
    """(module name, enclosing function or None) of every import in a module."""
    out = []

    def visit(node, fn):
        for ch in ast.iter_child_nodes(node):
            f = ch.name if isinstance(ch, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(ch, ast.Import):
                out.extend((a.name, fn) for a in ch.names)
            elif isinstance(ch, ast.ImportFrom):
                out.append((ch.module or "", fn))
            visit(ch, f)

    visit(tree, None)
    return out


def _py(path):
    return ast.parse(open(path).read(), filename=path)


def test_package_does_not_import_or_include_the_oracle():
    for path in glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True):
        for mod, _ in _imports(_py(path)):
            assert mod.split(".")[0] != "oracle", (path, mod)
    for path in glob.glob(os.path.join(PKG, "csrc", "*")):
        if not path.endswith((".cu", ".cuh", ".h", ".cpp")):
            continue
        for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', open(path).read()):
            assert "oracle" not in inc, (path, inc)
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', open(path).read()):
            assert "oracle" not in inc, (path, inc)


def test_oracle_does_not_import_or_include_the_package():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        for mod, _ in _imports(_py(path)):
            assert mod.split(".")[0] != "paper_2407_10797_gb300", (path, mod)
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.c")) + glob.glob(os.path.join(ROOT, "oracle", "*.h")):
        for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', open(path).read()):
            assert inc in {"complex.h", "math.h", "stdint.h", "stdlib.h", "string.h", "omp.h", "stdio.h",
                           "float.h"}, (path, inc)


def test_scripts_run_the_oracle_only_in_their_baseline_and_smoke_functions():
    # build() compiles the C oracle (building the checker, not running it)
    allowed = {"bench.py": {"oracle_sample", "run_reference"}, "__graft_entry__.py": {"build", "smoke"}}
    for name, fns in allowed.items():
        uses = [(mod, fn) for mod, fn in _imports(_py(os.path.join(ROOT, name))) if mod.split(".")[0] == "oracle"]
        assert uses, name
        for mod, fn in uses:
            assert fn in fns, (name, mod, fn)
