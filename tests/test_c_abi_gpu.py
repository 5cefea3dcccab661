"""The C ABI on its own: a plain C program (tests/c_abi_example.c) that uses
only gfc.h, the CUDA runtime and libgfc.so evaluates the bubble on a grid;
its output matches the oracle."""
import os
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1205_0752_gb300 as gfc  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_plain_c_program(tmp_path):
    lib = gfc.library_path()
    gfc.load_library()                       # builds libgfc.so if needed
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "c_abi_example")
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    subprocess.check_call([nvcc, os.path.join(HERE, "c_abi_example.c"), "-I", os.path.join(ROOT, "include"),
                           "-L", libdir, "-lgfc", "-Xlinker", f"-rpath,{libdir}", "-o", exe])
    m, n, nr, na = 8, 6, 256, 64
    out = subprocess.run([exe, str(m), str(n), str(nr), str(na)], capture_output=True, text=True,
                         timeout=120, check=True).stdout.split("\n")
    rows = [ln.split() for ln in out if ln and not ln.startswith("stats")]
    G = np.empty(m * n, dtype=np.complex128)
    for i, j, re, im in rows:
        G[int(i) * n + int(j)] = complex(float(re), float(im))
    x = oracle.grid_points(-8.0, 4.0, -4.0, 4.0, m, n)
    ref = oracle.eval_points({"kind": "scalar", "m2": 1.0},
                             dict(dim=4, mu2=1.0, n_radial=nr, n_angular=na), x)
    tau = 1e-3 * np.max(np.abs(ref))
    assert np.max(np.abs(G - ref) / np.maximum(np.abs(ref), tau)) < 1e-10
    stats = [ln for ln in out if ln.startswith("stats")][0].split()
    assert int(stats[1]) == m * n and int(stats[3]) >= 2
