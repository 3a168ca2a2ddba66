"""Run a few force-kernel launches on one workload, for profiling with ncu.

    python -m paper_1208_3444_b300.profile_force --workload grid32 --prec comp --launches 1

Prints the CUDA-event duration of each force-kernel launch (meaningless under
a profiler, which serialises and replays kernels).
"""
import argparse
import os
import sys

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
    a = p.parse_args()
    ic = workload(a.workload)
    sim = B.Simulation(ic.m, ic.eps, LCDM, 1.0, prec=PRECS[a.prec])
    try:
        sim.set_state(ic.x)
        sim.profile_forces(True)
        for _ in range(a.launches):
            sim.forces()
        ms, n = sim.profile_read()
    finally:
        sim.close()
    print(f"{a.workload} N={ic.N} prec={a.prec}: {n} launches, {ms / max(n, 1):.3f} ms each")


if __name__ == "__main__":
    main()
