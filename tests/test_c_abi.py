"""The boundary is a C ABI: a C99 program (gcc, -pedantic -Werror) includes
include/overlap.h, links liboverlap.so and calls the host-only entry points; its output
agrees with the oracle (Zolotarev coefficients, Sec. 3) and with NumPy (the host
numerics), and a bad argument comes back as OVL_EINVAL. The Python binding's ctypes
structures have the C layout, field by field, and its function signatures the header's
argument kinds, position by position. No GPU calls."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from oracle import zolotarev as zo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stdio.h>
#include <string.h>
#include "overlap.h"

int main(void) {
  double om[8], sg[8], de, lo, hi, w[3], z[18], a[18];
  const double d[4] = {2.0, 3.0, 4.0, 5.0}, e[3] = {1.0, 0.5, 0.25};
  int i;
  if (ovl_zolotarev_coeffs(8, 0.15, 2.6, om, sg, &de) != OVL_OK) return 1;
  for (i = 0; i < 8; ++i) printf("%.17g %.17g\n", om[i], sg[i]);
  printf("%.17g\n", de);
  if (ovl_host_tridiag_extremes(4, d, e, &lo, &hi) != OVL_OK) return 2;
  printf("%.17g %.17g\n", lo, hi);
  /* [[2, i, 0], [-i, 2, 0], [0, 0, 5]] as interleaved (re, im), row-major */
  memset(a, 0, sizeof(a));
  a[0] = 2.0; a[3] = 1.0; a[7] = -1.0; a[8] = 2.0; a[16] = 5.0;
  if (ovl_host_eigh(3, a, w, z) != OVL_OK) return 3;
  printf("%.17g %.17g %.17g\n", w[0], w[1], w[2]);
  printf("%d\n", (int)ovl_zolotarev_coeffs(0, 0.15, 2.6, om, sg, &de));
  printf("%s\n", ovl_version());
  return 0;
}
"""


@pytest.fixture(scope="module")
def c_program(tmp_path_factory):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1501_01855_gb300 import build
    lib = build.build()
    d = tmp_path_factory.mktemp("cabi")
    src = d / "t.c"
    src.write_text(C_SRC)
    exe = d / "t"
    libdir = os.path.dirname(lib)
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           str(src), "-L", libdir, "-loverlap", "-Wl,-rpath," + libdir, "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


def test_c_program_calls_the_library(c_program):
    r = subprocess.run([c_program], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    lines = r.stdout.strip().splitlines()
    om = np.array([float(l.split()[0]) for l in lines[:8]])
    sg = np.array([float(l.split()[1]) for l in lines[:8]])
    de = float(lines[8])
    o2, s2, d2 = zo.zolotarev(8, 0.15, 2.6)
    assert np.allclose(om, o2, rtol=1e-11, atol=0) and np.allclose(sg, s2, rtol=1e-11, atol=0)
    assert abs(de - d2) <= 1e-6 * d2 + 5e-15
    lo, hi = map(float, lines[9].split())
    T = np.diag([2.0, 3.0, 4.0, 5.0]) + np.diag([1.0, 0.5, 0.25], 1) + np.diag([1.0, 0.5, 0.25], -1)
    ev = np.linalg.eigvalsh(T)
    assert abs(lo - ev[0]) <= 1e-13 and abs(hi - ev[-1]) <= 1e-13
    w = np.array(list(map(float, lines[10].split())))
    assert np.allclose(w, [1.0, 3.0, 5.0], atol=1e-14)
    assert int(lines[11]) == -1                      # OVL_EINVAL
    assert lines[12].startswith("liboverlap")


def test_ctypes_structs_match_the_c_layout(tmp_path):
    """The binding's ctypes mirrors of ovl_params and ovl_solve_info have the C compiler's
    size and every field's offset (a drifted field would pass every later parameter
    shifted): a C program prints sizeof and offsetof for each field the binding names."""
    import ctypes
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1501_01855_gb300 import binding as B
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "overlap.h"', "int main(void) {"]
    for st in (B.ovl_params, B.ovl_solve_info):
        cname = st.__name__
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in st._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for st in (B.ovl_params, B.ovl_solve_info):
        cname = st.__name__
        assert int(out[cname]) == ctypes.sizeof(st), cname
        for f, _ in st._fields_:
            assert int(out["%s.%s" % (cname, f)]) == getattr(st, f).offset, (cname, f)


def _c_kind(decl):
    decl = decl.strip()
    if "*" in decl or "[" in decl:
        return "ptr"
    decl = re.sub(r"\b(const|unsigned)\b", "", decl).split()
    base = " ".join(decl[:-1]) if len(decl) > 1 else decl[0]
    return {"int": "int", "double": "double", "long long": "longlong", "size_t": "size_t"}.get(base, base)


def _ctypes_kind(t):
    import ctypes
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "ptr"
    return {ctypes.c_int: "int", ctypes.c_double: "double", ctypes.c_longlong: "longlong",
            ctypes.c_size_t: "size_t"}.get(t, repr(t))


def test_binding_signatures_match_the_header():
    """Every function the binding loads has, in include/overlap.h, the same number of
    arguments and the same kind (int, double, long long, pointer) in each position, and the
    same kind of result; a mismatch would pass garbage on both x86 and Arm."""
    from paper_1501_01855_gb300 import binding as B
    hdr = open(os.path.join(ROOT, "include", "overlap.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    protos = {}
    for m in re.finditer(r"([A-Za-z_][A-Za-z_0-9 \*]*?)\b((?:ovl|overlap|eigsumr)_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", hdr):
        ret, name, args = m.group(1), m.group(2), m.group(3)
        args = [] if args.strip() in ("", "void") else [a for a in args.split(",")]
        protos[name] = ("ptr" if "*" in ret else _c_kind(ret + " x").replace("ovl_status", "int"), [_c_kind(a) for a in args])
    for name, (res, argt) in B._SIGS.items():
        assert name in protos, name
        cres, cargs = protos[name]
        assert len(cargs) == len(argt), (name, cargs, argt)
        assert [_ctypes_kind(t) for t in argt] == cargs, (name, cargs)
        assert _ctypes_kind(res) == cres, (name, cres, res)


def test_binding_constants_match_the_header(tmp_path):
    """Status codes, element types, precisions, solvers and the profiler class count that
    the binding copies from include/overlap.h have the header's values."""
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1501_01855_gb300 import binding as B
    names = [n for n in dir(B) if re.fullmatch(r"OVL_[A-Z0-9_]+", n) and isinstance(getattr(B, n), int)]
    assert len(names) >= 18
    body = "\n".join('  printf("%s %%d\\n", (int)%s);' % (n, n) for n in names)
    src = tmp_path / "consts.c"
    src.write_text('#include <stdio.h>\n#include "overlap.h"\nint main(void) {\n%s\n  return 0;\n}\n' % body)
    exe = tmp_path / "consts"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for n in names:
        assert int(out[n]) == getattr(B, n), n
    assert set(B.STATUS_NAMES) == {getattr(B, n) for n in names if n.startswith("OVL_E") or n == "OVL_OK"}
