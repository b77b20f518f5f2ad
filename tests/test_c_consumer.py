"""The C ABI used from C: a plain C program compiled against include/hopf.h
and linked with libhopf_gb300.so checks defaults, validation and an empty
batch (no device work)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_links_and_validates(tmp_path):
    from paper_1712_08226_gb300 import build
    lib = build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(lib)
    cuda_lib = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")
    exe = str(tmp_path / "abi_consumer")
    cmd = [cc, "-std=c99", "-O1", "-Wall", "-Werror", os.path.join(ROOT, "tests", "c", "abi_consumer.c"),
           "-I", os.path.join(ROOT, "include"), "-L", libdir, "-l:" + os.path.basename(lib),
           "-Wl,-rpath," + libdir, "-Wl,-rpath," + cuda_lib, "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = os.pathsep.join(p for p in (libdir, cuda_lib, env.get("LD_LIBRARY_PATH", "")) if p)
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.stdout, r.stderr)
