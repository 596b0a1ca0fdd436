"""libpart.so used from plain C (tests/c_client/part_client.c), with no
Python and no torch on the path: built with gcc against include/part.h.
On the host it checks the host-only calls; on the GPU it runs one FP64
Boris + TSC + deposit step with cudaMalloc'd buffers, and the test compares
that step with the oracle (1e-12, as the parity tests)."""
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2602_23434_b300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "part_client.c")
OUT = os.path.join(ROOT, "_build", "part_client")


@pytest.fixture(scope="module")
def client():
    lib = build()
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    libdir = os.path.dirname(lib)
    subprocess.check_call([
        "gcc", "-O2", "-std=c11", "-I", os.path.join(ROOT, "include"),
        "-I", "/usr/local/cuda/include", "-o", OUT, SRC,
        "-L", libdir, "-lpart", "-L", "/usr/local/cuda/lib64", "-lcudart",
        f"-Wl,-rpath,{libdir}", "-Wl,-rpath,/usr/local/cuda/lib64"])
    return OUT


def _run(client, *args):
    r = subprocess.run([client, *args], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return r.stdout.splitlines()


def test_c_client_host_calls(client):
    out = _run(client, "host")
    assert out[0] == "brick 8 8 8 nkeys 2097152"
    assert out[1].startswith("workspace ") and int(out[1].split()[1]) > 0
    assert out[2].startswith("bad_dim 1 ") and "dim" in out[2]


@pytest.mark.gpu
def test_c_client_step_matches_the_oracle(client):
    N, n = 3001, 16
    lines = _run(client, "step", str(N), "97")
    vals = {}
    for ln in lines:
        k, v = ln.split(" ", 1)
        vals.setdefault(k, []).append(v)
    x0 = np.array(vals["x0"], dtype=np.float64).reshape(3, N)
    u0 = np.array(vals["u0"], dtype=np.float64).reshape(3, N)
    x1 = np.array(vals["x1"], dtype=np.float64).reshape(3, N)
    u1 = np.array(vals["u1"], dtype=np.float64).reshape(3, N)
    dep = np.array(vals["dep"], dtype=np.float64).reshape(3, n ** 3)
    assert int(vals["launches"][0]) > 0
    og = O.make_grid(3, (n, n, n))
    xi, ui, _, _ = O.init_particles(og, N, 97, 0.1)
    assert np.array_equal(x0, xi)                      # device draws, bit-exact positions
    assert np.max(np.abs(u0 - ui) / np.maximum(np.abs(ui), 0.1)) <= 1e-14
    f = np.zeros((6, n ** 3))
    f[0], f[5] = 0.01, 1.0
    perm = O.stable_sort(O.keys(og, (8, 8, 8), x0))    # the step sorts first
    xr, ur, F, xo = O.boris_step(og, O.TSC, f, x0[:, perm], u0[:, perm], None, 1.0, 0.05, True)
    d = x1 - xr
    d -= 2.0 * np.round(d / 2.0)
    assert np.max(np.abs(d)) <= 2e-12
    assert np.max(np.abs(u1 - ur)) <= 1e-12 * np.max(np.abs(ur))
    dref = O.deposit(og, O.TSC, xo, F)
    dabs = O.deposit(og, O.TSC, xo, np.abs(F))
    assert np.max(np.abs(dep - dref) / np.maximum(dabs, 1e-300)) <= 1e-12
