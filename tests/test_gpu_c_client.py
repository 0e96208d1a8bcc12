"""The whole path from a plain C program (tests/c_abi_device.c): CUDA
runtime allocations, the C ABI and nothing else; plain FP64 and batched
F16X3 C_l of the same sources agree within 1e-5."""
import os
import shutil
import subprocess

import pytest

from paper_2509_25110_gb300 import build, gcamb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_client_runs_the_batched_path(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    libdir = os.path.dirname(gcamb.LIB_PATH)
    cudalib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                    if os.path.exists(os.path.join(d, "libcudart.so"))), None)
    if cudalib is None:
        pytest.skip("no shared CUDA runtime")
    exe = str(tmp_path / "c_abi_device")
    r = subprocess.run([cc, "-std=c99", "-D_DEFAULT_SOURCE", "-Wall", "-Wextra", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c_abi_device.c"),
                        "-L", libdir, "-lgcamb", "-L", cudalib, "-lcudart", "-lm",
                        "-Wl,-rpath," + libdir + ":" + cudalib, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
    print(out.stdout.strip())
