"""The boundary is a C ABI: include/rbffd.h compiles as strict C99, and a
plain C program (no C++, no Python, no torch) links librbffd.so, resolves
every function the header declares and calls the ones that need no GPU.
No GPU needed."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rbffd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbffd_[a-z0-9_]+)\s*\(", src)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_plain_c_program_uses_the_library(tmp_path):
    from paper_1404_0812_gb300 import _lib
    _lib.load()
    libdir = os.path.dirname(_lib.library_path())
    names = _declared()
    refs = ",\n    ".join(f"(void (*)(void)){n}" for n in names)
    src = f"""
#include "rbffd.h"
#include <stdio.h>
#include <string.h>

/* every declared function, resolved at link time */
static void (*const all_functions[])(void) = {{
    {refs}
}};

int main(void) {{
    rbffd_build_opts o;
    unsigned i;
    for (i = 0; i < sizeof(all_functions) / sizeof(all_functions[0]); ++i)
        if (!all_functions[i]) return 10;
    rbffd_build_opts_default(&o);
    if (o.kernel != RBFFD_IMQ || o.kappa_target != 1e12 || o.eps_tol != 1e-4) return 11;
    if (strcmp(rbffd_status_str(RBFFD_OK), "ok") != 0) return 12;
    /* argument checks answer before any device work */
    if (rbffd_memory_pool_config(-1) != RBFFD_EINVAL) return 13;
    if (rbffd_fp64_peak(NULL, NULL) != RBFFD_EINVAL) return 14;
    printf("%u functions\\n", (unsigned)(sizeof(all_functions) / sizeof(all_functions[0])));
    return 0;
}}
"""
    c = tmp_path / "use_rbffd.c"
    c.write_text(src)
    inc = os.path.join(ROOT, "include")
    # the header alone, as strict C99
    subprocess.run(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                    "-I", inc, "-x", "c", os.path.join(inc, "rbffd.h")], check=True)
    exe = tmp_path / "use_rbffd"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", inc, str(c), "-o", str(exe),
                    "-L", libdir, "-lrbffd", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert out.stdout.strip() == f"{len(names)} functions"
