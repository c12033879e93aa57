"""The C ABI library loads (no GPU needed), exports every entry point that
include/thermo.h declares, and its host-only checks return the documented
status codes without touching a device."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "thermo.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(thermo_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2410_06850_gb300 import build, thermo
    build.build()
    return thermo.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "thermo_solve" in names and len(names) >= 16
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2410_06850_gb300",
                                                                      "libthermo.so")],
                         capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n


def test_binding_covers_header():
    from paper_2410_06850_gb300 import thermo
    assert sorted(thermo.EXPORTED) == _declared()


def test_struct_layouts_match_c(tmp_path):
    from paper_2410_06850_gb300 import thermo
    prog = tmp_path / "lay.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "thermo.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(thermo_options),'
                    ' offsetof(thermo_options, omega), offsetof(thermo_options, check_every),'
                    ' sizeof(thermo_solve_info), offsetof(thermo_solve_info, rel_res_true),'
                    ' offsetof(thermo_solve_info, status));return 0;}\n')
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    o, si = thermo.thermo_options, thermo.thermo_solve_info
    assert vals == [C.sizeof(o), o.omega.offset, o.check_every.offset, C.sizeof(si),
                    si.rel_res_true.offset, si.status.offset]


def test_default_options_host_only(L):
    from paper_2410_06850_gb300 import thermo
    o = thermo.default_options((256, 256, 256))  # coarsest 8^3 cells x 17 = 8,704 unknowns
    assert o.levels == 4 and o.block == 4
    assert list(o.nvec)[:4] == [4, 8, 17, 17]
    assert list(o.group)[1:4] == [2, 2, 2]
    o = thermo.default_options((128, 128, 128))  # coarsest 4^3 cells x 17 = 1,088 unknowns
    assert o.levels == 4 and list(o.nvec)[:4] == [4, 8, 17, 17]
    o = thermo.default_options((1024, 1024, 1024))
    assert o.levels == 6 and list(o.nvec)[:6] == [4, 8, 17, 17, 17, 17]
    o = thermo.default_options((32, 32, 32))
    assert o.levels == 2 and list(o.nvec)[:2] == [4, 17]
    with pytest.raises(thermo.ThermoError):
        thermo.default_options((30, 32, 32))


def test_host_argument_checks_need_no_gpu(L):
    from paper_2410_06850_gb300 import thermo
    ctx = C.c_void_p()
    g = (C.c_int * 3)(8, 8, 8)
    h = (C.c_double * 3)(0.125, 0.125, 0.125)
    assert L.thermo_create(g, h, None, None, None, None, None, C.byref(ctx)) == thermo.EINVAL
    assert L.thermo_create(None, None, None, None, None, None, None, None) == thermo.EINVAL
    assert L.thermo_last_error(None) == b"null context"
    L.thermo_destroy(None)
    assert L.thermo_set_density(None, None, 3.0, 1e-3, 1.0) == thermo.EINVAL
    assert L.thermo_solve(None, None, None, 1e-8, None) == thermo.EINVAL


def test_tpfa_and_resample_argument_checks_need_no_gpu(L):
    """The context-free entry points reject bad arguments before any launch."""
    from paper_2410_06850_gb300 import thermo
    g = (C.c_int * 3)(4, 4, 4)
    bad = (C.c_int * 3)(4, 0, 4)
    h = (C.c_double * 3)(0.25, 0.25, 0.25)
    fake = C.c_void_p(256)  # never dereferenced: every call below fails its checks first
    assert L.thermo_tpfa_apply(g, h, None, fake, fake, fake, None) == thermo.EINVAL
    assert L.thermo_tpfa_apply(bad, h, fake, fake, fake, C.c_void_p(512), None) == thermo.EINVAL
    assert L.thermo_tpfa_apply(g, h, fake, fake, fake, fake, None) == thermo.EINVAL  # t == y
    assert L.thermo_tpfa_rhs(g, h, fake, 0.5, 1.0, fake, fake, 0.0, fake, None) == thermo.EINVAL  # p < 1
    assert L.thermo_tpfa_sensitivity(g, h, fake, 3.0, 1e-3, 1.0, 1.0, fake, fake, 0.0, None, fake, fake,
                                     None) == thermo.EINVAL
    assert L.thermo_tpfa_conductivity(0, fake, 3.0, 1e-3, 1.0, fake, None) == thermo.EINVAL
    assert L.thermo_tpfa_conductivity(8, fake, 3.0, 0.0, 1.0, fake, None) == thermo.EINVAL  # kmin = 0
    gf = (C.c_int * 3)(6, 8, 8)
    assert L.thermo_resample(g, fake, gf, C.c_void_p(512), 0, None) == thermo.EINVAL  # 6 / 4 not an integer
    gf2 = (C.c_int * 3)(8, 8, 8)
    assert L.thermo_resample(g, fake, gf2, C.c_void_p(512), 3, None) == thermo.EINVAL  # kind
    assert L.thermo_resample(g, fake, gf2, fake, 0, None) == thermo.EINVAL  # in == out
