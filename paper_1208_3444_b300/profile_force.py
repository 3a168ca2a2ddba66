"""Run a few launches of one all-pairs kernel on one workload, for profiling
with ncu.

    python -m paper_1208_3444_b300.profile_force --workload grid32 --prec comp --launches 1
    python -m paper_1208_3444_b300.profile_force --op vjp --workload grid32 --launches 1
    python -m paper_1208_3444_b300.profile_force --periodic 1.0 --workload grid32 --launches 1
    python -m paper_1208_3444_b300.profile_force --op jvp --workload grid32 --launches 1
    python -m paper_1208_3444_b300.profile_force --op adjoint --workload grid32 --launches 2
    python -m paper_1208_3444_b300.profile_force --op vjp --periodic 1.0 --workload grid32 --launches 1
    python -m paper_1208_3444_b300.profile_force --op ensemble --launches 1
    python -m paper_1208_3444_b300.profile_force --op spectrum --launches 1
    python -m paper_1208_3444_b300.profile_force --op diagnostics --workload grid32 --launches 1

--op adjoint runs colatus_adjoint_forward over --launches steps (checkpoints
every step) and colatus_adjoint_backward (the equal-mass VJP for equal-mass
workloads); --op force runs colatus_forces (the force kernel, or with --periodic L the
Ewald real-space and k-space kernels); --op vjp runs colatus_force_vjp with a
seeded co-vector; --op jvp runs tangent steps of 64 single-tracer tangents
(one JVP launch each); --op ensemble runs force evaluations of the
64-realisation ensemble (--workload is ignored); --op spectrum runs
colatus_velocity_spectrum on a seeded device series of 2000 records of 64
tracers (Hann window, detrended; --workload is ignored); --op diagnostics
runs colatus_diagnostics (the O(N^2) potential energy and the moments).  Prints the CUDA-event duration of the force or VJP
kernel (meaningless under a profiler, which serialises and replays kernels).
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1208_3444_b300 import binding as B  # noqa: E402
from paper_1208_3444_b300 import inputs  # noqa: E402

LCDM = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
PRECS = {"fp32": B.FP32, "comp": B.FP32_COMP, "fp64": B.FP64}


def workload(name):
    if name == "grid16":
        return inputs.grid16()
    if name == "grid32":
        return inputs.grid32()
    if name.startswith("uniform"):
        return inputs.uniform(int(name[len("uniform"):]), 3)
    if name.startswith("plummer"):
        return inputs.plummer_clusters(int(name[len("plummer"):]), 9)
    raise ValueError(name)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="grid32",
                   help="grid16 | grid32 | uniform<N> | plummer<N>")
    p.add_argument("--prec", default="comp", choices=sorted(PRECS))
    p.add_argument("--launches", type=int, default=1)
    p.add_argument("--op", default="force", choices=["force", "vjp", "jvp", "adjoint", "ensemble", "spectrum",
                            "diagnostics"])
    p.add_argument("--periodic", type=float, default=0.0, help="box side L (0: isolated)")
    a = p.parse_args()
    if a.op == "ensemble":
        ics = inputs.ensemble(64, seed=5)
        ens = B.Ensemble(np.array([c.N for c in ics]), np.concatenate([c.m for c in ics]),
                         [c.eps for c in ics], LCDM, 1.0)
        try:
            ens.set_state(np.concatenate([c.x for c in ics]), np.concatenate([c.v for c in ics]))
            for _ in range(a.launches):
                ens.forces()
            ens.synchronize()
        finally:
            ens.close()
        print(f"ensemble: 64 realisations, {a.launches} force evaluations")
        return
    if a.op == "spectrum":
        import torch
        g = torch.Generator(device="cuda").manual_seed(11)
        v = torch.randn((2000, 64, 3), device="cuda", dtype=torch.float32, generator=g)
        out = torch.empty((64, 1001), device="cuda", dtype=torch.float64)
        for _ in range(a.launches):
            B.colatus_velocity_spectrum(v, inputs.lcdm_tau(2000), "hann", True, out=out)
        torch.cuda.synchronize()
        print(f"spectrum: T=2000, 64 tracers, {a.launches} calls")
        return
    ic = workload(a.workload)
    sim = B.Simulation(ic.m, ic.eps, LCDM, 1.0, prec=PRECS[a.prec])
    try:
        sim.set_state(ic.x, ic.v)
        if a.periodic:
            sim.set_periodic(a.periodic)
        if a.op == "jvp":
            sim.tangent_init(inputs.tracers(ic.N, 64, 7), a.launches)
            sim.tangent_step(inputs.lcdm_tau(2000), a.launches)
            sim.synchronize()
            print(f"jvp {a.workload} N={ic.N}: {a.launches} tangent steps of 64 tangents")
            return
        if a.op == "adjoint":
            sim.adjoint_forward(inputs.lcdm_tau(2000), a.launches, 1)
            gv = np.zeros((ic.N, 3))
            gv[inputs.tracers(ic.N, 64, 7)] = 1.0
            sim.adjoint_backward(None, gv)
            sim.synchronize()
            print(f"adjoint {a.workload} N={ic.N} prec={a.prec}: {a.launches} steps forward and back")
            return
        if a.op == "diagnostics":
            for _ in range(a.launches):
                d = sim.diagnostics()
            print(f"diagnostics {a.workload} N={ic.N} prec={a.prec}: {a.launches} calls, W={d['W']:.9e}")
            return
        w = np.random.default_rng(1).standard_normal((ic.N, 3))
        sim.profile_forces(True)
        for _ in range(a.launches):
            if a.op == "vjp":
                sim.force_vjp(w)
            else:
                sim.forces()
        ms, n = sim.profile_read(vjp=a.op == "vjp")
    finally:
        sim.close()
    print(f"{a.op} {a.workload} N={ic.N} prec={a.prec} periodic={a.periodic}: {n} launches, "
          f"{ms / max(n, 1):.3f} ms each")


if __name__ == "__main__":
    main()
