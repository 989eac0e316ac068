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


def _cuda_home():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return d
    return None


@pytest.mark.gpu
def test_c_client_runs_the_path_on_the_gpu(gpu_lib, tmp_path):
    """tests/c_gpu_client.c: cudaMalloc'd fields, upload, z = a*b and its
    reverse mode through the C ABI, checked against the oracle's C library."""
    import oracle
    import synth
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda = _cuda_home()
    if cc is None or cuda is None:
        pytest.skip("no C compiler or CUDA headers")
    lib = su3s.lib_path()
    syn, ora = synth.build(), oracle.build()
    libdirs = [os.path.dirname(lib), os.path.dirname(syn), os.path.dirname(ora),
               os.path.join(cuda, "lib64")]
    exe = str(tmp_path / "c_gpu_client")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), os.path.join(HERE, "c_gpu_client.c"), "-o", exe,
           "-L", os.path.dirname(lib), "-lsu3s", syn, ora, "-L", os.path.join(cuda, "lib64"),
           "-lcudart", "-lm"] + ["-Wl,-rpath," + d for d in libdirs]
    subprocess.check_call(cmd)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok ")
