"""Accuracy of the force sweep configuration against the FP64 oracle:
N in {2^16, 2^18, 2^21}, uniform and clustered bodies (eps = 1e-3), FP32
plain / compensated / FP64 on the GPU, on seeded target rows (4096 rows; 1024
at 2^21).  Prints the rel-RMS error of every case (run with -s to see it)."""
import numpy as np
import pytest

import oracle
from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

pytestmark = pytest.mark.gpu

LCDM_D = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
TOL = {B.FP32: 1e-5, B.FP32_COMP: 1e-6, B.FP64: 1e-11}
NAME = {B.FP32: "fp32", B.FP32_COMP: "comp", B.FP64: "fp64"}


@pytest.mark.parametrize("lg", [16, 18, 21])
@pytest.mark.parametrize("workload", ["uniform", "plummer"])
def test_sweep_case(lg, workload):
    N = 1 << lg
    ic = inputs.uniform(N, 3) if workload == "uniform" else inputs.plummer_clusters(N, 9)
    nrows = 1024 if lg >= 21 else 4096
    rows = np.sort(np.random.default_rng(1000 + lg).choice(N, nrows, replace=False))
    ref = oracle.forces(ic.x, ic.m, ic.eps, rows=rows)
    scale = np.mean(np.linalg.norm(ref, axis=1))
    for prec in (B.FP32, B.FP32_COMP, B.FP64):
        if prec == B.FP64 and lg > 18:
            continue                      # one FP64 force at 2^21 takes over a minute
        sim = B.Simulation(ic.m, ic.eps, LCDM_D, 1.0, prec=prec)
        try:
            sim.set_state(ic.x)
            got = sim.forces()[rows]
        finally:
            sim.close()
        err = float(np.sqrt(np.mean(np.sum((got - ref) ** 2, axis=1))) / scale)
        print(f"sweep N=2^{lg} {workload} {NAME[prec]}: rel-RMS {err:.2e}")
        assert err < TOL[prec]
