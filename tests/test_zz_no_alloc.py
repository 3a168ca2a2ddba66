"""The allocation-free force entry point, colatus_forces_noalloc, against the
context-based colatus_forces.

Some callers cannot call cudaMalloc: code that runs inside another framework's
memory pool or under a fixed device-memory budget, and latency-bound loops that
must not pay cudaMalloc's implicit device synchronisation.  They use
colatus_forces_noalloc, whose scratch is one fixed static device array shared
by every call.  Two calls in a row, with different sizes, must each match
colatus_forces within the FP32 force tolerance of the other tests (RMS over
bodies of the difference, relative to the mean |acc|: 1e-5), and so must each
match the FP64 oracle, which shares no code with either.  This file is
collected after every other test file.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
TOL = 1e-5


def rel_rms(a, b):
    return float(np.sqrt(np.mean(np.sum((a - b) ** 2, axis=1))) /
                 np.mean(np.linalg.norm(b, axis=1)))


def with_context(ic, a, G):
    sim = B.Simulation(ic.m, ic.eps, LCDM, a, prec=B.FP32, G=G)
    try:
        sim.set_state(ic.x)
        return sim.forces()
    finally:
        sim.close()


def without_allocation(ic, a, G):
    import torch
    pos = torch.tensor(np.concatenate([ic.x, ic.m[:, None]], axis=1), dtype=torch.float32,
                       device="cuda")
    out = torch.full((ic.N, 3), float("nan"), dtype=torch.float32, device="cuda")
    B.colatus_forces_noalloc(pos, ic.eps, G, a, out, stream=torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy().astype(np.float64)


def test_two_calls_in_a_row_match_colatus_forces():
    rng = np.random.default_rng(77)
    first = inputs.ICs(x=inputs.f32(rng.random((5000, 3))), v=np.zeros((5000, 3)),
                       m=inputs.f32(rng.lognormal(0.0, 0.5, 5000) / 5000), eps=0.01, name="random")
    second = inputs.grid32()
    for ic, a, G in ((first, 0.5, 1.3), (second, inputs.A_START, 1.0)):
        got = without_allocation(ic, a, G)
        ref = with_context(ic, a, G)
        assert np.all(np.isfinite(got))
        assert rel_rms(got, ref) < TOL
        exact = oracle.forces(ic.x, ic.m, ic.eps, G) / a ** 3
        assert rel_rms(got, exact) < TOL


def test_largest_size_with_lognormal_masses_matches_oracle():
    # N = 32768, the size limit, on the wide-tile path; lognormal masses take
    # the general-mass kernel.  Checked against the FP64 oracle on 2048 rows.
    rng = np.random.default_rng(78)
    N = 32768
    ic = inputs.ICs(x=inputs.f32(rng.random((N, 3))), v=np.zeros((N, 3)),
                    m=inputs.f32(rng.lognormal(0.0, 0.5, N) / N), eps=1e-3, name="lognormal32768")
    rows = np.sort(rng.choice(N, 2048, replace=False))
    for _ in range(2):
        got = without_allocation(ic, 0.7, 1.0)
        exact = oracle.forces(ic.x, ic.m, ic.eps, 1.0, rows=rows) / 0.7 ** 3
        assert np.all(np.isfinite(got))
        assert rel_rms(got[rows], exact) < TOL


def test_rejects_buffers_it_cannot_use():
    # every check below returns before any launch
    import torch
    N = 1000
    buf = torch.zeros(N * 4 + 1, dtype=torch.float32, device="cuda")
    out = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
    f = B.lib().colatus_forces_noalloc
    # pos not 16-byte aligned
    assert f(buf.data_ptr() + 4, N, 0.01, 1.0, 1.0, out.data_ptr(), None) == B.E_ARG
    # host memory instead of device memory
    host = np.zeros((N, 4), dtype=np.float32)
    hout = np.zeros((N, 3), dtype=np.float32)
    assert f(host.ctypes.data, N, 0.01, 1.0, 1.0, out.data_ptr(), None) == B.E_ARG
    assert f(buf.data_ptr(), N, 0.01, 1.0, 1.0, hout.ctypes.data, None) == B.E_ARG
    # the output was not touched, and a good call still works afterwards
    assert torch.count_nonzero(out).item() == 0
    pos = buf[:N * 4].view(N, 4)
    pos[:, :3] = torch.rand((N, 3), device="cuda")
    pos[:, 3] = 1.0 / N
    B.colatus_forces_noalloc(pos, 0.01, 1.0, 1.0, out)
    assert torch.isfinite(out).all().item()
    with pytest.raises(ValueError):
        B.colatus_forces_noalloc(pos, 0.01, 1.0, 1.0, out[:N - 1])


def test_rejects_more_bodies_than_the_static_scratch_holds():
    import torch
    N = 32769
    pos = torch.zeros((N, 4), dtype=torch.float32, device="cuda")
    out = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(B.ColatusError) as e:
        B.colatus_forces_noalloc(pos, 0.01, 1.0, 1.0, out)
    assert e.value.status == B.E_ARG
