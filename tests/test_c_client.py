"""The C ABI from plain C: tests/c_client.c, compiled as strict C99 against
include/colatus.h and linked with libcolatus.so, no Python or C++ in between.

* CPU: the header compiles as C99 with every warning an error, the program
  links, and without a GPU it fails cleanly with COLATUS_E_CUDA from
  colatus_init (exit status 2 + 2) and the library's message.  The host-only
  self-tests of the pair-once tables run through the C ABI and return the
  same figures as through the Python binding.
* GPU: the Eq. 1 acceleration, 3 KDK steps with FP32 compensated forces, (t,
  a) and the diagnostics, read back through the C program's output file,
  against the FP64 oracle (force rel-RMS 1e-6, positions 1e-5 max abs,
  velocities RMS-relative 1e-5, a to 1e-12, W to 1e-5 and K to 1e-4, as for
  the Python path).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import build as libbuild
from paper_1208_3444_b300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LCDM = oracle.Cosmology(0.0, 0.3, 0.0, 0.7, 1.0)   # the program's fixed cosmology
TAU = inputs.lcdm_tau(2000)
NDIAG = 16


def compile_client(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = libbuild.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "c_client")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_client.c"), "-L", libdir, "-lcolatus",
           "-Wl,-rpath," + libdir, "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def write_input(path, x, v, m, eps, a_start, tau, nsteps):
    with open(path, "wb") as f:
        np.array([len(m), nsteps], dtype=np.int64).tofile(f)
        np.array([eps, a_start, tau], dtype=np.float64).tofile(f)
        np.asarray(m, dtype=np.float64).tofile(f)
        np.asarray(x, dtype=np.float32).tofile(f)
        np.asarray(v, dtype=np.float32).tofile(f)


def read_output(path, N):
    raw = open(path, "rb").read()
    f32 = np.frombuffer(raw[:9 * N * 4], dtype=np.float32).reshape(3, N, 3)
    tail = np.frombuffer(raw[9 * N * 4:], dtype=np.float64)
    assert tail.size == 2 + NDIAG
    return f32[0], f32[1], f32[2], tail[0], tail[1], tail[2:]


def test_c_client_compiles_as_c99_and_fails_cleanly_without_gpu(tmp_path):
    exe = compile_client(tmp_path)
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the run is checked by the GPU test")
    ic = inputs.grid8()
    write_input(tmp_path / "in.bin", ic.x, ic.v, ic.m, ic.eps, inputs.A_START, TAU, 1)
    r = subprocess.run([exe, str(tmp_path / "in.bin"), str(tmp_path / "out.bin")],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 2 + 2, (r.returncode, r.stderr)     # COLATUS_E_CUDA from colatus_init
    assert "colatus_init" in r.stderr and "status 2" in r.stderr


def test_c_client_runs_the_table_self_tests(tmp_path):
    from paper_1208_3444_b300 import binding as B
    exe = compile_client(tmp_path)
    r = subprocess.run([exe, "selftest"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    lines = dict((ln.split()[0], [int(t) for t in ln.split()[1:]]) for ln in r.stdout.splitlines())
    keys = ("tiles", "tile_pairs", "ctas", "row_segments", "column_slots")
    want = B.colatus_selftest_sym_tables(32768, 2048, 32, 147, 11, 14)
    assert lines["sym"] == [want[k] for k in keys]
    want = B.colatus_selftest_ens_sym_tables([1028, 4096, 4097, 32675], 592, 11, 14)
    assert lines["ens"] == [want[k] for k in keys]
    assert lines["sym"][:2] == [16, 136]


@pytest.mark.gpu
def test_c_client_matches_oracle(tmp_path):
    exe = compile_client(tmp_path)
    ic = inputs.grid16(critical=True)
    n = 3
    write_input(tmp_path / "in.bin", ic.x, ic.v, ic.m, ic.eps, inputs.A_START, TAU, n)
    r = subprocess.run([exe, str(tmp_path / "in.bin"), str(tmp_path / "out.bin")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    acc, x, v, t, a, diag = read_output(tmp_path / "out.bin", ic.N)

    ref_acc = oracle.forces(ic.x, ic.m, ic.eps) / inputs.A_START ** 3
    err = np.sqrt(np.mean(np.sum((acc - ref_acc) ** 2, axis=1))) / np.mean(np.linalg.norm(ref_acc, axis=1))
    assert err < 1e-6

    ref = oracle.run(ic.x, ic.v, ic.m, ic.eps, 1.0, LCDM, inputs.A_START, TAU, n, "kdk")
    assert np.abs(x - ref["x"]).max() < 1e-5
    rms = lambda d: float(np.sqrt(np.mean(np.sum(d ** 2, axis=1))))  # noqa: E731
    assert rms(v - ref["v"]) < 1e-5 * rms(ref["v"])
    a_ref = ref["schedule"]["a"][-1]
    assert a == pytest.approx(a_ref, rel=1e-12)
    assert t == pytest.approx(n * TAU, rel=1e-12)
    d = oracle.diagnostics(ref["x"], ref["v"], ic.m, a_ref, ic.eps, 1.0, LCDM)
    assert diag[0] == pytest.approx(d["K"], rel=1e-4)   # K
    assert diag[1] == pytest.approx(d["W"], rel=1e-5)   # W
    assert diag[15] == n                                # steps taken
