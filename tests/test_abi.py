"""The C ABI: libbl.so builds for sm_103a, loads, and exports every function include/bl.h declares
(no GPU needed: nothing here launches a kernel).  Also the host-side strategy grammar (Table 1)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(bl_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2412_08264_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_call_sequence():
    names = declared_functions()
    for required in ["bl_problem_create", "bl_lower_solve", "bl_hessian_solve", "bl_ritz_update",
                     "bl_hypergrad", "bl_problem_destroy", "bl_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_exported_symbol(lib):
    from paper_2412_08264_gb300 import _lib as L
    assert set(L.EXPORTS) == declared_functions()


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the option structs have the sizes and field offsets the C compiler gives them."""
    import shutil
    import subprocess
    from paper_2412_08264_gb300 import _lib as L
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"bl_pair_desc": L.PairDesc, "bl_reg_desc": L.RegDesc, "bl_lbfgs_opts": L.LbfgsOpts,
               "bl_krylov_opts": L.KrylovOpts, "bl_recycle_opts": L.RecycleOpts, "bl_solve_info": L.SolveInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bl.h"', "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for cname, cls in mirrors.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)


def test_invalid_arguments_fail_without_gpu(lib):
    """Argument validation happens before any CUDA call."""
    from paper_2412_08264_gb300 import _lib as L
    lib2 = L.load()
    out = ctypes.c_void_p()
    assert lib2.bl_problem_create(None, 1, None, None, None, None, ctypes.byref(out)) == L.BL_EINVAL
    pd = (L.PairDesc * 1)(L.PairDesc(8, 8, 1.5, 2))
    rd = L.RegDesc(L.BL_REG_FOE, 2, 4, 0, 0.01, 1e-6, L.BL_FP32, 4, 10)     # even filter size
    dummy = ctypes.c_void_p(16)
    assert lib2.bl_problem_create(pd, 1, ctypes.byref(rd), dummy, dummy, None, ctypes.byref(out)) == L.BL_EINVAL
    assert b"filter_size" in lib2.bl_last_error()
    rd = L.RegDesc(L.BL_REG_FOE, 2, 5, 0, 0.01, 1e-6, L.BL_FP32, 60, 60)    # W too wide
    assert lib2.bl_problem_create(pd, 1, ctypes.byref(rd), dummy, dummy, None, ctypes.byref(out)) == L.BL_EINVAL
    pd = (L.PairDesc * 1)(L.PairDesc(8, 8, 1.5, 5))                          # blur radius > 4
    rd = L.RegDesc(L.BL_REG_FOE, 2, 5, 0, 0.01, 1e-6, L.BL_FP32, 4, 10)
    assert lib2.bl_problem_create(pd, 1, ctypes.byref(rd), dummy, dummy, None, ctypes.byref(out)) == L.BL_EINVAL


def test_library_refuses_to_load_when_missing(tmp_path):
    from paper_2412_08264_gb300 import _lib as L
    saved = L._lib
    L._lib = None
    try:
        with pytest.raises(RuntimeError, match="not found"):
            L.load(str(tmp_path / "libbl.so"))
    finally:
        L._lib = saved


@pytest.mark.parametrize("acr,kind,size,side,nsc", [
    ("Ritz-S", "ritz", "S", "R", False), ("HRitz-L", "hritz", "L", "R", False),
    ("RGen-L(R)", "rgsv", "L", "R", False), ("RGen-M(L)-NSC", "rgsv", "M", "L", True),
    ("RGen-S(M)", "rgsv", "S", "M", False), ("none", "none", "S", "R", False)])
def test_strategy_grammar(acr, kind, size, side, nsc):
    from paper_2412_08264_gb300.strategy import parse
    st = parse(acr)
    assert (st.kind, st.size, st.side, st.nsc) == (kind, size, side, nsc)
    if kind != "none":
        assert parse(st.acronym()) == st


@pytest.mark.parametrize("bad", ["Ritz-S(R)", "RGen-L", "Eig-S", "Ritz-X", "Ritz-S-NSC", "GSVD-L(R)"])
def test_strategy_grammar_rejects(bad):
    from paper_2412_08264_gb300.strategy import parse
    with pytest.raises(ValueError):
        parse(bad)


def test_static_jw_validates_before_any_cuda_call(tmp_path):
    """bl_jw_fp32_static rejects sizes beyond its fixed scratch and invalid options before it makes a
    CUDA call: run in a child process that sees no GPU, with placeholder pointers that are never
    dereferenced (a regression that reached a launch would fail there with BL_ECUDA, not touch a GPU)."""
    import subprocess
    import sys
    script = r'''
import ctypes, sys
sys.path.insert(0, %r)
from paper_2412_08264_gb300 import _lib as L
lib = L.load()
d = ctypes.c_void_p(256)
cases = [
    # 2048 x 2048 with 48 7x7 filters: 64 * 64 tiles * 2400 values > 524288
    ((d, d, 2048, 2048, d, 48, 7, 0, 0.01, d, None), b"static scratch"),
    ((d, d, 64, 64, d, 4, 4, 0, 0.01, d, None), b"filter_size"),
    ((d, d, 0, 64, d, 4, 5, 0, 0.01, d, None), b"sizes"),
    ((d, d, 64, 64, d, 65, 5, 0, 0.01, d, None), b"n_filters"),
    ((d, d, 64, 64, d, 4, 5, 7, 0.01, d, None), b"phi"),
    ((d, d, 64, 64, d, 4, 5, 0, 0.0, d, None), b"phi_eps"),
    ((None, d, 64, 64, d, 4, 5, 0, 0.01, d, None), b"null"),
]
for args, word in cases:
    st = lib.bl_jw_fp32_static(*args)
    msg = lib.bl_last_error()
    assert st == L.BL_EINVAL, (args, st, msg)
    assert word in msg, (word, msg)
print("ok")
''' % ROOT
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    from paper_2412_08264_gb300 import build
    build.build()
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
