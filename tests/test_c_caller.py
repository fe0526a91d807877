"""libsu3 from a plain C99 program (tests/c/su3_c_caller.c): no Python or PyTorch in the process
that calls the C ABI. On CPU the program compiles under -std=c99 -pedantic -Werror (the CUDA
runtime header as a system header) and links against libsu3, the CUDA runtime, the oracle and the
input generator; on a GPU it runs su3_mult (device buffers) and su3_mult_host (pageable buffers on
the path the library picks and on the staged path, pinned buffers), NATIVE and F32PAIR, and checks
every result against the FP64 oracle within 1e-13."""
import os
import subprocess

import pytest

import paper_2103_00571_gb300 as su3
from paper_2103_00571_gb300 import build as su3_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "su3_c_caller.c")


def compile_caller(out_dir):
    import oracle
    import su3_inputs
    libs = [os.path.dirname(su3.library_path()), os.path.dirname(oracle.build()),
            os.path.dirname(su3_inputs.build()), su3_build.cuda_lib_dir()]
    cuda_root = os.path.dirname(os.path.dirname(os.path.realpath(su3_build.nvcc())))
    exe = os.path.join(str(out_dir), "su3_c_caller")
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           "-isystem", os.path.join(cuda_root, "include"), SRC, "-o", exe]
    for d in libs:
        cmd += ["-L", d, "-Wl,-rpath," + d]
    cmd += ["-lsu3", "-lsu3oracle", "-lsu3gen", "-lcudart", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_caller_builds_and_links(tmp_path):
    assert os.access(compile_caller(tmp_path), os.X_OK)


@pytest.mark.gpu
@pytest.mark.parametrize("L", [8, 13])
def test_c_caller_matches_oracle(tmp_path, L):
    """L=8 (4,096 sites) and L=13 (28,561 sites: ragged against every tile size) from C."""
    exe = compile_caller(tmp_path)
    r = subprocess.run([exe, str(L)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c caller ok" in r.stdout
    assert r.stdout.count("max abs err") == 8  # 2 arithmetics x (device, pageable, pageable staged, pinned)
