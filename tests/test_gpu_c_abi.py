"""The C ABI from C: tests/c_abi_example.c (host buffers only, no CUDA headers, no
Python in the caller) is built with gcc against libgmaf.so and its Picard step is
compared with the oracle's on the same inputs (FP64: loads 1e-7; mixed: 1e-5)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def example(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2511_06824_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path_factory.mktemp("c_abi") / "c_abi_example")
    subprocess.run(["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_example.c"), "-L", libdir, "-lgmaf",
                    f"-Wl,-rpath,{libdir}", "-o", exe], check=True)
    return exe


def run(exe, nth, nz, precision):
    r = subprocess.run([exe, str(nth), str(nz), str(precision)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    out = {}
    for line in r.stdout.splitlines():
        f = line.split()
        out[f[0]] = f[1:]
    return int(out["status"][0]), int(out["status"][2]), np.array(out["loads"], float), \
        np.array(out["G"], float), np.array(out["state"], float)


def load_err(a, b):
    out = 0.0
    for part in (slice(0, 6), slice(6, 12)):
        x, y = a[part], b[part]
        out = max(out, float(np.max(np.abs(x - y) / np.maximum(np.abs(y), 1e-3 * np.linalg.norm(y)))))
    return out


@pytest.mark.parametrize("nth,nz,precision", [(128, 64, 0), (256, 128, 1)])
def test_c_caller_picard_step_matches_oracle(example, nth, nz, precision):
    st, iters, loads, G, state = run(example, nth, nz, precision)
    assert st == 0 and iters > 0
    phys = np.array([1e-2, 4e-2, 2e-5, 0.04, 5.0, 2e7, 1e5])
    tex = np.array([1, 5e-4, 5e-6, 0.2, 1e-4, 2e-4])
    st0 = np.array([2e-6, -1e-6, 3e-6, 1e-6, 1e-5, 0.0, -2e-5, 0.0])
    o = oracle.picard_step(nth, nz, phys, tex, st0, st0[:4] - 2e-8, 2.78e-4,
                           np.array([25.0, -10.0, 4.0, 3.0]), 2e-8, 1e-6, eps=1e-12)
    assert o["status"] == oracle.OK
    assert load_err(loads, o["loads"]) <= (1e-7 if precision == 0 else 1e-5)
    np.testing.assert_allclose(G, o["G"], rtol=1e-6, atol=1e-6 * np.abs(o["G"]).max())
    ds, dso = state - st0, o["state"] - st0
    assert np.linalg.norm(ds - dso) <= 1e-4 * np.linalg.norm(dso)
