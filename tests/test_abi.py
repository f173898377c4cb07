"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/crmc.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "crmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cr_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2109_07527_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("cr_init", "cr_sweep", "cr_md_forces", "cr_state"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2109_07527_gb300 import crmc
    assert sorted(crmc.EXPORTS) == _declared()


def test_strerror_names_every_code(lib):
    lib.cr_strerror.restype = ctypes.c_char_p
    seen = set()
    for code in range(0, -10, -1):
        s = lib.cr_strerror(code).decode()
        assert s and s != "unknown error"
        seen.add(s)
    assert len(seen) == 10


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the ABI structs match the C layout compiled from the header."""
    import subprocess
    from paper_2109_07527_gb300 import crmc
    structs = {"cr_system": crmc.cr_system, "cr_mu_ions": crmc.cr_mu_ions, "cr_sweep_stats": crmc.cr_sweep_stats,
               "cr_state_view": crmc.cr_state_view, "cr_info": crmc.cr_info, "cr_mlp": crmc.cr_mlp,
               "cr_load_args": crmc.cr_load_args, "cr_batch_packed": crmc.cr_batch_packed,
               "cr_counters": crmc.cr_counters, "cr_train_cfg": crmc.cr_train_cfg,
               "cr_ungrouped": crmc.cr_ungrouped, "cr_device_buffers": crmc.cr_device_buffers}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "crmc.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            cf = "global" if f == "global_" else f
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {cf}));')
    lines.append('  printf("cr_trial %zu\\n", sizeof(cr_trial));')
    lines.append('  printf("cr_trial_da %zu\\n", sizeof(cr_trial_da));')
    for f in crmc.DA_DTYPE.names:
        lines.append(f'  printf("cr_trial_da.{f} %zu\\n", offsetof(cr_trial_da, {f}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
    assert int(got["cr_trial"]) == crmc.TRIAL_DTYPE.itemsize
    assert int(got["cr_trial_da"]) == crmc.DA_DTYPE.itemsize
    for f in crmc.DA_DTYPE.names:
        assert int(got[f"cr_trial_da.{f}"]) == crmc.DA_DTYPE.fields[f][1], f


def test_header_is_plain_c_and_cpp():
    """The boundary header compiles warning-free as strict C99 and as C++11
    (no C++-only constructs, no torch or CUDA types in the signatures)."""
    import subprocess
    h = os.path.join(ROOT, "include", "crmc.h")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c", h])
    subprocess.check_call(["g++", "-std=c++11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c++",
                           h])
    import re
    code = re.sub(r"//[^\n]*", "", re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S))
    for banned in ("torch", "at::", "cudaStream_t", "#include <cuda"):
        assert banned not in code, banned
