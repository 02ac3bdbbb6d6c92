"""A plain-C client (tests/c_client/solve_demo.c) uses the library through
include/pot3d.h alone: it compiles as C99 and links on the CPU; on the GPU
it solves with host arrays, evaluates the field and checks the FP64
residual and the inner-face field itself."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "solve_demo.c")


def build_demo(out_dir):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    from paper_1709_01126_gb300 import _build

    lib = _build.build()
    libdir = os.path.dirname(lib)
    exe = os.path.join(str(out_dir), "solve_demo")
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I",
                           os.path.join(ROOT, "include"), SRC, "-L", libdir, "-lpot3d",
                           "-Wl,-rpath," + libdir, "-lm", "-o", exe])
    return exe


def test_c_client_compiles_and_links(tmp_path):
    assert os.path.exists(build_demo(tmp_path))


@pytest.mark.gpu
@pytest.mark.parametrize("dims", [(12, 17, 37), (9, 40, 130)])
def test_c_client_solves(tmp_path, dims):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = build_demo(tmp_path)
    r = subprocess.run([exe] + [str(d) for d in dims], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("status 0 ")
