"""Every entry point declared in include/fstat.h, called with NULL handles and
pointers and zero sizes, refuses without a device call and without touching
memory: status-returning calls give FS_EINVAL with a message that names the
call (the destroy calls accept NULL and return FS_OK), the int-returning
queries give -1.  The calls run in a child process so that a crash fails this
test instead of ending the test session."""
import json
import os
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SWEEP = textwrap.dedent(r'''
    import ctypes as C, json, re, sys
    sys.path.insert(0, ROOT)
    from paper_2407_10797_gb300 import fstat
    L = fstat.load()
    src = open(ROOT + "/include/fstat.h").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decls = re.findall(r"FS_API\s+([\w\s\*]+?)\b(fs_\w+)\s*\(([^)]*)\)\s*;", src)
    SCALAR = {"int": C.c_int, "int64_t": C.c_int64, "uint64_t": C.c_uint64, "double": C.c_double,
              "float": C.c_float, "fs_precision": C.c_int, "fs_tdi": C.c_int}
    out = []
    for ret, name, params in decls:
        ats = []
        for p in (q.strip() for q in params.split(",")):
            if not p or p == "void":
                continue
            if "*" in p or p.split()[0] in ("cudaStream_t",):
                ats.append(C.c_void_p)
                continue
            words = p.replace("const", "").split()
            ats.append(SCALAR[" ".join(words[:-1])])
        f = getattr(L, name)
        f.argtypes = ats
        kind = "str" if "char" in ret else ("i64" if "int64_t" in ret else "int")
        f.restype = {"str": C.c_char_p, "i64": C.c_int64, "int": C.c_int}[kind]
        L.fs_last_error.restype = C.c_char_p
        r = f(*[None if a is C.c_void_p else 0 for a in ats])
        msg = (L.fs_last_error() or b"").decode()
        out.append([name, ret.strip(), r.decode() if isinstance(r, bytes) else r, msg])
    print(json.dumps(out))
''')


def test_every_entry_point_refuses_null_and_zero_arguments():
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + SWEEP], capture_output=True, text=True,
                       timeout=300, env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr[-3000:]
    rows = json.loads(r.stdout.strip().splitlines()[-1])
    names = [n for n, _, _, _ in rows]
    assert len(names) == len(set(names)) and len(names) >= 50
    for name, ret, value, msg in rows:
        if name == "fs_last_error":
            assert isinstance(value, str)
        elif name in ("fs_plan_destroy", "fs_graph_destroy", "fs_mlp_destroy"):
            assert value == 0, name
        elif ret.endswith("fs_status"):
            assert value == -1, (name, value, msg)
            # the message names the call (fs_plan_create_tdi reports through fs_plan_create)
            head = msg.split(":")[0]
            assert head and name.startswith(head), (name, msg)
        else:
            assert value == -1, (name, value)
