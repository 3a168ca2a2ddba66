"""Force-kernel throughput sweep: N in {2^16, 2^18, 2^21}, uniform and
clustered (Plummer spheres, lognormal masses) bodies, FP32 plain, FP32
compensated and FP64, eps = 1e-3.

    python -m paper_1208_3444_b300.sweep [--sizes 16,18,21] [--fp64-max 18]

Times each force launch with CUDA events (library-side, on the launching
stream) after one warm-up launch, 10 launches per case by default, and
prints one JSON line per case with the median launch: interactions/s,
interactions/SM/clk at the GPU's maximum clock, and the fraction of the
20-flop convention roofline (12.8 interactions/SM/clk).
FP64 is skipped above 2^fp64-max bodies (at 2^21 one FP64 force takes over a
minute).  Accuracy against the FP64 oracle is checked by the test suite.
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1208_3444_b300 import binding as B  # noqa: E402
from paper_1208_3444_b300 import inputs  # noqa: E402

LCDM = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
PRECS = (("fp32", B.FP32), ("comp", B.FP32_COMP), ("fp64", B.FP64))


def case(ic, prec, launches):
    """Milliseconds of each of `launches` force launches after a warm-up."""
    sim = B.Simulation(ic.m, ic.eps, LCDM, 1.0, prec=prec)
    try:
        sim.set_state(ic.x)
        sim.forces()                      # warm-up (module load, segment buffers)
        sim.profile_forces(True)
        out = []
        for _ in range(launches):
            sim.forces()
            ms, n = sim.profile_read()
            out.append(ms / n)
        sim.profile_forces(False)
    finally:
        sim.close()
    return out


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--sizes", default="16,18,21", help="log2 N values")
    p.add_argument("--fp64-max", type=int, default=18)
    p.add_argument("--launches", type=int, default=10)
    a = p.parse_args()
    import torch
    props = torch.cuda.get_device_properties(0)
    sms, mhz = props.multi_processor_count, 2032.0
    for lg in (int(s) for s in a.sizes.split(",")):
        N = 1 << lg
        for wname, ic in (("uniform", inputs.uniform(N, 3)), ("plummer", inputs.plummer_clusters(N, 9))):
            for pname, prec in PRECS:
                if pname == "fp64" and lg > a.fp64_max:
                    continue
                t = case(ic, prec, a.launches)
                ms = float(np.median(t))
                ips = float(N) * N / (ms * 1e-3)
                per = ips / (sms * mhz * 1e6)
                print(json.dumps({"N": N, "workload": wname, "prec": pname, "launches": len(t),
                                  "ms_per_force": ms, "ms_min": min(t), "ms_max": max(t),
                                  "interactions_per_s": ips, "int_per_sm_per_clk": per,
                                  "frac_of_fp32_roofline": per / 12.8}), flush=True)


if __name__ == "__main__":
    main()
