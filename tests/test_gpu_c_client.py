"""The C ABI used from a plain C program (include/brev.h, the CUDA runtime
and nothing else): compiled with gcc against libbrev.so and the oracle's C
library, run, and checked against the oracle inside the program."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_uses_the_abi(brev_lib, oracle_lib, tmp_path):
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    gcc = shutil.which("gcc")
    assert gcc, "gcc is needed to build the C client"
    libdir = os.path.dirname(brev_lib.LIB_PATH)
    oracledir = os.path.join(ROOT, "oracle")
    exe = str(tmp_path / "brev_c_client")
    cmd = [gcc, "-O2", "-std=c99", os.path.join(ROOT, "tests", "c", "brev_c_client.c"),
           "-I", os.path.join(ROOT, "include"), "-I", oracledir, "-I", os.path.join(cuda, "include"),
           "-L", libdir, "-L", oracledir, "-L", os.path.join(cuda, "lib64"),
           f"-Wl,-rpath,{libdir}:{oracledir}:{os.path.join(cuda, 'lib64')}",
           "-l:" + os.path.basename(brev_lib.LIB_PATH), "-loracle", "-lcudart", "-o", exe]
    subprocess.run(cmd, check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "c client ok" in r.stdout
