"""The C ABI without a GPU: the library builds, loads, exports every symbol
that include/ac.h declares, and rejects invalid arguments before touching the
device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ac():
    from paper_0710_0736_gb300 import build
    build.build()
    from paper_0710_0736_gb300 import ac as mod
    return mod


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ac_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_match_header(ac):
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(ac.lib, name), f"{name} declared but not exported"
    assert declared == set(ac.EXPORTS)


def test_default_params(ac):
    p = ac.ac_default_params(stream=None)
    assert (p.tol, p.nu1, p.nu2, p.max_cycles, p.coarse_min, p.precision) == (1e-10, 2, 2, 200, 4, ac.AC_FP64)


@pytest.mark.parametrize("field,value", [
    ("width", 0), ("height", -3), ("height", 70000), ("refine", -1), ("refine", 5), ("n_phases", 1), ("n_phases", 9), ("eps", 0.0), ("tau", -1.0),
    ("lambda_", -0.5), ("tol", 0.0), ("nu1", -1), ("max_cycles", 0), ("coarse_min", 0), ("precision", 7),
])
def test_create_rejects_bad_params(ac, field, value):
    p = ac.ac_default_params(width=8, height=8, n_phases=3, eps=2.0, tau=4.0, stream=None)
    p.lambda_ = 1.0
    setattr(p, field, value)
    ctx = C.c_void_p()
    assert ac.lib.ac_create(C.byref(ctx), C.byref(p)) == ac.AC_ERR_ARG
    assert ctx.value is None
    assert ac.ac_last_error()


def test_null_arguments(ac):
    assert ac.lib.ac_step(None, 1, None) == ac.AC_ERR_ARG
    assert ac.lib.ac_set_image(None, None, 0) == ac.AC_ERR_ARG
    assert ac.lib.ac_project_simplex(None, None, 4, 9, None) == ac.AC_ERR_ARG
    assert ac.lib.ac_project_simplex(None, None, -1, 4, None) == ac.AC_ERR_ARG
    ac.ac_destroy(None)  # accepted


def test_oracle_is_not_linked(ac):
    """The product library must not depend on the oracle."""
    import subprocess
    out = subprocess.run(["nm", "-D", ac._LIB_PATH], capture_output=True, text=True).stdout
    assert "or_" not in " ".join(l.split()[-1] for l in out.splitlines() if l.split())


def _header_signatures():
    """(return type, parameter types) of every ac_* declaration in include/."""
    sigs = {}
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for ret, name, args in re.findall(r"([A-Za-z_][A-Za-z0-9_ \*]*?)\b(ac_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", txt,
                                          flags=re.S):
            args = " ".join(args.split())
            params = [] if args in ("", "void") else [a.strip() for a in args.split(",")]
            # a parameter's type: the declaration without its name
            types = [re.sub(r"\s*\b[A-Za-z_][A-Za-z0-9_]*$", "", p) for p in params]
            sigs[name] = (" ".join(ret.split()), types)
    return sigs


def _c_kind(t):
    t = t.replace("const ", "").strip()
    if "*" in t:
        return "ptr"
    return {"int": "i32", "unsigned": "u32", "int64_t": "i64", "double": "f64", "void": "void"}[t]


def _ctypes_kind(ct):
    if ct is None:
        return "void"
    if ct in (C.c_void_p, C.c_char_p) or (isinstance(ct, type) and issubclass(ct, C._Pointer)):
        return "ptr"
    if ct is C.c_int:
        return "i32"
    if ct is C.c_uint:
        return "u32"
    if ct in (C.c_int64, C.c_longlong):
        return "i64"
    if ct is C.c_double:
        return "f64"
    raise AssertionError(f"unexpected ctypes type {ct}")


def test_binding_signatures_match_header(ac):
    """The ctypes binding passes every call the arguments its declaration
    names: the same count, and pointers, 32- and 64-bit integers and doubles
    in the same places (a drift here would hand the library garbage)."""
    sigs = _header_signatures()
    assert set(sigs) == set(ac.EXPORTS)
    for name, (ret, types) in sigs.items():
        f = getattr(ac.lib, name)
        got = [_ctypes_kind(t) for t in (f.argtypes or [])]
        assert got == [_c_kind(t) for t in types], name
        assert _ctypes_kind(f.restype) == _c_kind(ret), name


def test_struct_layouts_match_header(ac, tmp_path):
    """Every struct the ABI passes by pointer has the same size and field
    offsets in the ctypes binding as in include/ac.h compiled as plain C."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"ac_params": ac.ac_params, "ac_stats": ac.ac_stats, "ac_profile": ac.ac_profile,
               "ac_batch_stats": ac.ac_batch_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ac.h"', "int main(void) {"]
    for s, cls in structs.items():
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in cls._fields_:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {cf}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (l.split() for l in out if l.strip())}
    for s, cls in structs.items():
        assert got[(s, "size")] == C.sizeof(cls), s
        for f, _ in cls._fields_:
            assert got[(s, f)] == getattr(cls, f).offset, (s, f)


def test_constants_match_header(ac, tmp_path):
    """Every AC_* constant of the binding has the header's value (status
    codes, precisions, modes), and the profile classes are in the header's
    order."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "ac.h")).read(), flags=re.S)
    header = set(re.findall(r"\b(AC_[A-Z0-9_]+)\s*(?:=|,|\n|\})", txt)) - {"AC_H"}
    header = sorted(header | set(re.findall(r"#define[ \t]+(AC_[A-Z0-9_]+)[ \t]+\S", txt)))
    names = [n for n in header if hasattr(ac, n)]
    assert len(names) >= 20
    lines = ['#include <stdio.h>', '#include "ac.h"', "int main(void) {"]
    lines += [f'  printf("{n} %lld\\n", (long long)({n}));' for n in names]
    prof = [f"AC_PROF_{c.upper()}" for c in ac.PROF_CLASSES]
    lines += [f'  printf("{n} %lld\\n", (long long)({n}));' for n in prof + ["AC_PROF_COUNT"]]
    lines += ["  return 0;", "}"]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {a: int(b) for a, b in (l.split() for l in out if l.strip())}
    for n in names:
        assert getattr(ac, n) == got[n], n
    assert [got[n] for n in prof] == list(range(len(prof))) and got["AC_PROF_COUNT"] == len(prof)
