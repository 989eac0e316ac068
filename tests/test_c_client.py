"""The C ABI from C: tests/c_client.c is compiled as C99 with warnings as
errors against include/su3s.h, linked to the library and run.  It uses only
the host side of the ABI (no kernel is launched), so it runs without a GPU."""
import os
import shutil
import subprocess

import pytest

import paper_1710_09409_gb300 as su3s

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_c_client_builds_and_runs(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    su3s.load(build_if_missing=True)
    lib = su3s.lib_path()
    exe = str(tmp_path / "c_client")
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "c_client.c"),
                           "-o", exe, "-L", os.path.dirname(lib), "-lsu3s",
                           "-Wl,-rpath," + os.path.dirname(lib)])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok ")
