"""The C ABI from plain C.  tests/c_abi_example.c includes only the CUDA
runtime's C header and include/u1u1.h, allocates its fields with cudaMalloc
and runs the path: initial conditions, steps with fused detection, records,
standalone detection and diagnostics.  Without a GPU it must compile as
pedantic C11 and link against libu1u1.  On a GPU its printed results must
equal the Python binding's for the same parameters, bit for bit: the same
kernels run with the same launches.
"""
import os
import shutil
import subprocess

import pytest

import paper_2208_01525_gb300 as U
from paper_2208_01525_gb300 import build as B

SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c_abi_example.c")


def build_example(tmp_path) -> str:
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    U.lib()  # builds libu1u1.so if the sources are newer
    cuda_include = os.path.join(os.path.dirname(os.path.dirname(B.nvcc())), "include")
    obj, exe = str(tmp_path / "c_abi_example.o"), str(tmp_path / "c_abi_example")
    r = subprocess.run([gcc, "-std=c11", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", B.INCLUDE, "-I",
                        cuda_include, "-c", SRC, "-o", obj], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([B.nvcc(), "-o", exe, obj, "-L", B.OUT_DIR, "-lu1u1", "-Xlinker", f"-rpath={B.OUT_DIR}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_example_compiles_as_c11_and_links(tmp_path):
    assert os.access(build_example(tmp_path), os.X_OK)


@pytest.mark.gpu
def test_c_example_equals_the_python_binding(tmp_path):
    torch = pytest.importorskip("torch")
    side = 24
    r = subprocess.run([build_example(tmp_path), str(side)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    got = dict(kv.split("=") for kv in r.stdout.split())

    p = U.Params.cube(side, m=0.5, beta=1.0, eta0=1.0, eta_ref=1.0 + 0.1 * 32, seed=7, precision=U.FP32)
    lat = U.Lattice(p)
    lat.step(32, detect_every=16)
    recs, lost = lat.read_records(max_records=4)
    s = lat.detect_strings(tol=1)
    d = lat.diagnostics()
    n, cur = lat.current()
    torch.cuda.synchronize()
    assert int(got["records"]) == len(recs) == 2 and int(got["lost"]) == lost == 0
    assert int(got["n"]) == n == 32 and int(got["current"]) == cur
    for r_, (rs, rd) in enumerate(recs):
        assert int(got[f"rec{r_}_n"]) == rs["n"]
        assert int(got[f"rec{r_}_n_p"]) == rs["n_p"] and int(got[f"rec{r_}_n_q"]) == rs["n_q"]
        assert float(got[f"rec{r_}_energy"]) == rd["energy"]
    for k in ("n_p", "n_q", "n_pq_plaq", "n_pq_cell"):
        assert int(got[k]) == s[k], k
    assert float(got["xi_w"]) == s["xi_w"]
    assert float(got["energy"]) == d["energy"] and float(got["lag"]) == d["lag"]
    lat.close()
