"""CPU checks of the C-ABI boundary: the library builds, loads, and exports
every function include/dwfmg.h and include/dwfnet.h declare (no compute calls
without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = "".join(open(os.path.join(ROOT, "include", h)).read() for h in ("dwfmg.h", "dwfnet.h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:dwf_status|void|unsigned long long|const char\s*\*|char\s*\*)\s*\*?\s*(\w+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1205_2933_gb300 import build as B
    return str(B.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dwf_create", "dwf_apply", "mg_setup", "mg_solve", "dwf_pack", "dwf_unpack",
                     "dwf_strerror", "dwf_destroy", "mg_default_params", "net_create", "net_forward",
                     "net_loss_grad", "net_adam", "mg_vcycle_batch"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_host_only_calls(libpath):
    L = ctypes.CDLL(libpath)
    L.dwf_strerror.restype = ctypes.c_char_p
    assert L.dwf_strerror(0) == b"success"
    assert b"converge" in L.dwf_strerror(-4)
    from paper_1205_2933_gb300 import dwfmg as G
    p = G.mg_default_params()
    assert p.split == 1 and p.nu_post > 0 and 1 <= p.outer_restart <= 64 and p.setup_sweep_tol == 0.1
    # invalid arguments are rejected before any device work
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert G.lib().dwf_create(ctypes.byref(h), 1, ctypes.cast(d, ctypes.c_void_p), 0, 1.8, 0.1, None, 1, None) \
        == G.DWF_EINVAL
    assert G.lib().dwf_create(ctypes.byref(h), 0, ctypes.cast(d, ctypes.c_void_p), 8, 1.8, 0.1, None, 1, None) \
        == G.DWF_EINVAL
    assert G.lib().dwf_lattice(None, 0, ctypes.byref(h)) == G.DWF_EINVAL
    assert G.lib().dwf_apply(None, None, None, 0, 0, 1) == G.DWF_EINVAL
    assert G.lib().net_create(None, None, None) == G.DWF_EINVAL
    assert G.lib().net_adam(None, 1e-3, 0.9, 0.999, 1e-8) == G.DWF_EINVAL


def test_no_cpu_fallback_in_product_path():
    """The package never imports the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_1205_2933_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".c", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structs have the header's field offsets and sizes
    (a C program built with gcc from include/dwfmg.h prints them)."""
    from paper_1205_2933_gb300 import dwfmg as G
    structs = {"mg_params": G.mg_params, "mg_stats": G.mg_stats, "dwf_net_shape": G.dwf_net_shape}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dwfmg.h"', '#include "dwfnet.h"',
             'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        name, field, value = line.split()
        cls = structs[name]
        expect = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert int(value) == expect, (name, field, value, expect)


def test_environment_switches_are_documented():
    """Every environment variable the library reads is listed in the header."""
    csrc = os.path.join(ROOT, "paper_1205_2933_gb300", "csrc")
    used = set()
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cuh", ".h")):
            used |= set(re.findall(r'getenv\("([A-Z0-9_]+)"\)', open(os.path.join(csrc, f)).read()))
    header = open(os.path.join(ROOT, "include", "dwfmg.h")).read()
    assert used, "no switches found"
    missing = sorted(v for v in used if v not in header)
    assert not missing, missing
