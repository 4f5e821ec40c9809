"""The boundary is a plain C ABI: a C program (tests/c/abi_host_plan.c)
compiles against include/tn_gb300.h with a C compiler, links the library and
plans a circuit on the host.  No GPU is needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_plans_through_the_abi(tmp_path):
    import paper_2111_03011_gb300 as tn
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = os.path.dirname(tn.lib._name)
    exe = str(tmp_path / "abi_host_plan")
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-O1", os.path.join(ROOT, "tests", "c", "abi_host_plan.c"),
                    "-I", os.path.join(ROOT, "include"), "-L", lib, "-ltn_gb300", "-Wl,-rpath," + lib, "-lm",
                    "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert "c abi ok" in out.stdout
