#!/usr/bin/env python
"""Benchmark of the COLATUS hot path on B300: one KDK step of the 32^3 run.

A timed "step" is one pass of the whole path on the 32^3 workload (perturbed
grid, growing-mode velocities, eps = 0.02 spacing): the FP64 Friedmann
schedule, the FP32 all-pairs force with compensated accumulation, the fused
kick-drift epilogue with Hubble drag, and the 64-tracer record.

Prints ONE JSON line (rank 0).  ``value`` is pair interactions per second
(N^2 per step) over all ranks; ``roofline`` reports the force kernel against
the FP32-FMA/MUFU issue roofline (20 flops per interaction by convention;
256 FP32 flop/clk/SM); ``force_128cubed`` times the force alone at
N = 2^21 = 128^3; ``cpu_baseline`` times the FP64 oracle on a bounded sample
on this host's cores.  ``--impl reference`` times only the oracle.

Multi-GPU (torchrun): every rank runs an independent replica of the same
workload (weak scaling); the barrier and the max-over-ranks time are the
only communication.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairwise interactions/sec & % FP32/MUFU roofline at N=32³,128³; adjoint/fwd time"
UNIT = "interactions/s"
LCDM = dict(Omega_R=0.0, Omega_M=0.3, Omega_K=0.0, Omega_L=0.7, H0=1.0)
FLOPS_PER_INTERACTION = 20          # Nyland et al. convention
FP32_FLOP_PER_CLK_PER_SM = 256      # 128 FP32 lanes x FMA
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the 32^3 compensated equal-mass force kernel (the pair-once shape), from one
# ncu capture.  The figure is reported only while the launched kernel has the
# captured shape and its source files hash to the captured sources; otherwise
# traffic is null.
FORCE_KERNEL_TRAFFIC = {
    "bytes": 560128,
    "plan": dict(kind="force_sym_f32", threads=512, ipt=4, jt=2048, comp=True, eqm=True, nrcp=0),
    "template": "force_sym_f32_kernel<512, 4, 1, 1, 8, PlummerPair>",
    "sources": ('paper_1208_3444_b300/csrc/force_sym.cuh', 'paper_1208_3444_b300/csrc/force.cuh', 'paper_1208_3444_b300/csrc/common.cuh'),
    "sha256": "48db95745b2737294274299a46a4a1a42a1e03f396f9976f15ce4c687bdb924d",
}


def pair_lane_ops(plan, N):
    """FP32 lane-ops of the pair arithmetic per counted interaction (N^2 per
    force) for the launched force kernel: 11 (equal masses) or 12 per ordered
    pair; the pair-once form 14 or 16 per pair in the tile pairs it < jt and
    11 or 12 per ordered pair in the diagonal tiles, over the padded bodies."""
    eqm = plan.get("eqm")
    one, both = (11, 14) if eqm else (12, 16)
    t = plan["jt"]
    if plan.get("kind") == "force_sym_f32":
        n = -(-N // t)
        work = ((n * (n + 1) // 2 - n) * both + n * one) * float(t) * t
    else:
        npad = -(-N // max(t, plan["threads"] * plan["ipt"])) * max(t, plan["threads"] * plan["ipt"])
        work = one * float(npad) * npad
    return work / (float(N) * N)


def source_hash(paths):
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def force_traffic(plan):
    """The captured DRAM bytes per launch if `plan` (Simulation.force_plan())
    is the captured kernel built from the captured sources, else None."""
    t = FORCE_KERNEL_TRAFFIC
    same_shape = all(plan.get(k) == v for k, v in t["plan"].items())
    same_source = source_hash(t["sources"]) == t["sha256"]
    return (t["bytes"] if same_shape and same_source else None), same_shape, same_source


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="colatus", choices=["colatus", "reference"])
    p.add_argument("--no-128", action="store_true", help="skip the N = 128^3 force timing")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    return p.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in self.lines:
            f = [s.strip() for s in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), power=float(f[3]),
                                 hw=f[5], hwt=f[6], swt=f[7], swp=f[8]))
            except ValueError:
                continue
        if not rows:
            return None
        load = [r for r in rows if r["power"] > 200.0] or rows
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r["sm"] for r in load])),
                "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------ CPU baseline
def cpu_baseline(seconds, rows_per_call=2048):
    """The FP64 oracle (as it stands) on a bounded row sample of the 32^3
    workload: forces on random target rows against all 32^3 sources, repeated
    until about `seconds` of CPU time have been spent."""
    import oracle
    from paper_1208_3444_b300 import inputs
    ic = inputs.grid32()
    rng = np.random.default_rng(0)
    oracle.forces(ic.x, ic.m, ic.eps, rows=np.arange(64))        # start the thread pool
    cores = oracle.num_threads()

    def rate(budget, rows):
        done, calls = 0, 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget:
            oracle.forces(ic.x, ic.m, ic.eps, rows=np.sort(rng.choice(ic.N, rows, replace=False)))
            done += rows
            calls += 1
        dt = time.perf_counter() - t0
        return done * ic.N / dt, done, calls, dt

    value, done, calls, dt = rate(seconds, rows_per_call)
    oracle.set_threads(1)
    one, done1, _, dt1 = rate(max(1.0, seconds / 5), 128)
    oracle.set_threads(cores)
    cpu = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            cpu = next(l.split(":", 1)[1].strip() for l in f if l.startswith("model name"))
    except (OSError, StopIteration):
        pass
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "value_1_thread": one, "cpu": cpu,
            "sample": f"FP64 oracle forces on {done} random target rows ({calls} calls of "
                      f"{rows_per_call}) x all {ic.N} sources of the 32^3 workload ({dt:.1f} s) on "
                      f"{cores} threads; {done1} rows on 1 thread ({dt1:.1f} s)"}


# --------------------------------------------------------------- distributed
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate_throughput(ws, steps, pairs, ms_max):
    """Whole-job interactions/s: every rank ran `steps` steps of `pairs`
    interactions; the slowest rank's time (ms) bounds the job."""
    return ws * steps * float(pairs) / (ms_max * 1e-3)


def max_over_ranks(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ arms
def run_reference(args, ws, rank):
    if rank != 0:
        return None
    import oracle
    from paper_1208_3444_b300 import inputs
    ic = inputs.grid32()
    # 2048 target rows per step (the CPU baseline's call size): enough work
    # per call to keep every host core busy; 200 steps take a few seconds
    rows_per_step = 2048
    rng = np.random.default_rng(1)
    for _ in range(args.warmup):
        oracle.forces(ic.x, ic.m, ic.eps,
                      rows=np.sort(rng.choice(ic.N, rows_per_step, replace=False)))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.forces(ic.x, ic.m, ic.eps,
                      rows=np.sort(rng.choice(ic.N, rows_per_step, replace=False)))
    dt = time.perf_counter() - t0
    value = args.steps * rows_per_step * ic.N / dt
    sample = (f"each step: FP64 oracle forces on {rows_per_step} random target bodies x all "
              f"{ic.N} sources of the 32^3 workload")
    return {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "grid32 (N=32^3 perturbed grid), force rows sampled",
                       "N": ic.N},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def time_force_128(B, inputs, torch, launches=3):
    """FP32 force alone at N = 2^21 (uniform bodies), events around each launch."""
    ic = inputs.uniform(1 << 21, 11)
    st = torch.cuda.current_stream().cuda_stream
    assert st, "use a created stream, not the legacy default stream"
    sim = B.Simulation(ic.m, ic.eps, LCDM, 1.0, prec=B.FP32, stream=st)
    out = torch.empty((ic.N, 3), dtype=torch.float32, device="cuda")
    try:
        sim.set_state(ic.x)
        plan = sim.force_plan()
        sim.forces(out)
        sim.synchronize()
        sim.profile_forces(True)
        for _ in range(launches):
            sim.forces(out)
        ms, n = sim.profile_read()
        sim.profile_forces(False)
    finally:
        sim.close()
    return {"N": ic.N, "launches": n, "ms_per_launch": ms / n,
            "interactions_per_s": ic.N * ic.N * n / (ms * 1e-3), "prec": "fp32", "plan": plan}


def time_adjoint(B, inputs, torch, stream, nsteps=200, k=20):
    """Adjoint vs forward step time on the 32^3 workload (FP32 compensated), in
    the adjoint configuration: 200 KDK steps, checkpoints every 20.  Reports
    the adjoint step (one VJP + the transposed update, timed by events around
    those kernels) over the forward step, the backward wall time less the
    recomputed forces over the forward step, and the total including the
    recomputation."""
    ic = inputs.grid32()
    tau = inputs.lcdm_tau(2000)
    sim = B.Simulation(ic.m, ic.eps, LCDM, inputs.A_START, prec=B.FP32_COMP, scheme=B.KDK,
                       stream=stream.cuda_stream)
    try:
        sim.set_state(ic.x, ic.v)
        vplan = sim.vjp_plan()
        gv = np.zeros((ic.N, 3))
        gv[inputs.tracers(ic.N, 64, 7)] = 1.0
        # warm-up pass of the same shape: loads the adjoint kernels (lazy
        # module loading) and sizes the checkpoint buffers outside the timed region
        sim.adjoint_forward(tau, nsteps, k)
        sim.adjoint_backward(None, gv)
        sim.set_state(ic.x, ic.v)
        sim.step(tau, 3)
        sim.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        sim.profile_forces(True)
        ev[0].record(stream)
        sim.adjoint_forward(tau, nsteps, k)
        ev[1].record(stream)
        fwd = sim.profile_read_all()
        ev[2].record(stream)
        sim.adjoint_backward(None, gv)
        ev[3].record(stream)
        torch.cuda.synchronize()
        bwd = sim.profile_read_all()
        sim.profile_forces(False)
    finally:
        sim.close()
    f = ev[0].elapsed_time(ev[1]) / nsteps
    b = ev[2].elapsed_time(ev[3]) / nsteps
    rec = bwd["force"][0] / nsteps
    vjp = bwd["vjp"][0] / bwd["vjp"][1]
    # the adjoint step: one VJP and one transposed update per step (plus the
    # final VJP at x_0), each bracketed by events on the launching stream
    adj = (bwd["vjp"][0] + bwd["adjoint_update"][0]) / nsteps
    # FP32 lane-ops per interaction of the VJP kernel the adjoint ran: the
    # pair-once form takes 27 per pair in the tile pairs it < jt and 23 per
    # ordered pair in the diagonal tiles; the per-ordered-pair equal-mass form
    # 23, the general (scaled) form 25
    if vplan["kind"] == "vjp_sym_eqm_f32":
        t, nt = vplan["jt"], ic.N // vplan["jt"]
        ops = ((nt * (nt + 1) // 2 - nt) * 27 + nt * 23) * float(t * t) / (float(ic.N) * ic.N)
    else:
        ops = 23.0 if vplan["kind"] == "vjp_eqm_f32" else 25.0
    vrate = ic.N * ic.N / (vjp * 1e-3) / (torch.cuda.get_device_properties(0).multi_processor_count * 2.032e9)
    return {"N": ic.N, "steps": nsteps, "checkpoint_every": k, "prec": "fp32_comp", "vjp_plan": vplan,
            "forward_ms_per_step": f, "backward_ms_per_step": b,
            "recompute_ms_per_step": rec, "vjp_ms_per_launch": vjp,
            "update_ms_per_launch": bwd["adjoint_update"][0] / max(1, bwd["adjoint_update"][1]),
            "adjoint_step_ms": adj,
            "force_ms_per_launch": fwd["force"][0] / fwd["force"][1],
            "adjoint_step_over_forward_step": adj / f,
            "backward_minus_recompute_forces_over_forward": (b - rec) / f,
            "backward_total_over_forward": b / f,
            "vjp_interactions_per_sm_per_clk": vrate,
            "vjp_lane_ops_per_interaction": ops,
            "vjp_frac_of_lane_op_floor": vrate / (128.0 / ops),
            "vjp_floor_note": "FP32 lane-ops per interaction of the launched VJP kernel (vjp_plan) at "
                              "128 lane-ops/SM/clk"}


def time_ensemble(B, inputs, torch, stream, nsteps=48):
    """The 64-realisation ensemble (N_r log-uniform in [1024, 32768]): the
    autotuner picks the force kernel's CTA shape, then KDK steps under the
    library's captured 16-step graphs, aggregate throughput."""
    ics = inputs.ensemble(64, seed=5)
    Ns = np.array([ic.N for ic in ics])
    ens = B.Ensemble(Ns, np.concatenate([ic.m for ic in ics]), [ic.eps for ic in ics], LCDM,
                     inputs.A_START, stream=stream.cuda_stream)
    try:
        ens.set_state(np.concatenate([ic.x for ic in ics]), np.concatenate([ic.v for ic in ics]))
        tune_ms, shape = ens.autotune(3)      # the project's autotuner picks the CTA shape
        tau = inputs.lcdm_tau(2000)
        ens.step(tau, 16)
        ens.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ens.stats()["launches"]
        e0.record(stream)
        ens.step(tau, nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        st = ens.stats()
    finally:
        ens.close()
    ms = e0.elapsed_time(e1)
    pairs = float(np.sum(Ns.astype(float) ** 2))
    return {"realisations": len(ics), "N_total": int(Ns.sum()), "N_min": int(Ns.min()),
            "N_max": int(Ns.max()), "interactions_per_step": pairs, "steps": nsteps,
            "ms_per_step": ms / nsteps, "interactions_per_s": pairs * nsteps / (ms * 1e-3),
            "graph_launches": nsteps // 16, "kernel_launches": st["launches"] - l0,
            "autotune": {"shape": shape, "ms_per_force": [round(float(t), 4) for t in tune_ms],
                         "shapes": ["128x2, 4 CTAs/SM", "256x1, 4 CTAs/SM", "64x4, 8 CTAs/SM",
                                    "128x4 on 512-body tiles, every pair once, 4 CTAs/SM"]},
            "interactions_per_sm_per_clk": pairs * nsteps / (ms * 1e-3) /
            (torch.cuda.get_device_properties(0).multi_processor_count * 2.032e9),
            "frac_of_fp32_roofline": pairs * nsteps / (ms * 1e-3) /
            (torch.cuda.get_device_properties(0).multi_processor_count * 2.032e9) / 12.8}


def time_tangent(B, inputs, torch, stream, ntr=64, nsteps=2):
    """Tangent-linear propagation of 64 single-tracer perturbations through
    the 32^3 KDK steps (FP32): one JVP launch per step for all 64 tangents."""
    ic = inputs.grid32()
    tau = inputs.lcdm_tau(2000)
    sim = B.Simulation(ic.m, ic.eps, LCDM, inputs.A_START, prec=B.FP32, stream=stream.cuda_stream)
    try:
        sim.set_state(ic.x, ic.v)
        sim.tangent_init(inputs.tracers(ic.N, ntr, 7), nsteps + 1)
        sim.tangent_step(tau, 1)
        sim.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.tangent_step(tau, nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        growth = sim.tangent_growth()
    finally:
        sim.close()
    ms = e0.elapsed_time(e1) / nsteps
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    tint = float(ic.N) * ic.N * ntr
    return {"N": ic.N, "tangents": ntr, "ms_per_step": ms,
            "tangent_interactions_per_s": tint / (ms * 1e-3),
            "tangent_interactions_per_sm_per_clk": tint / (ms * 1e-3) / (nsm * 2.032e9),
            "finite": bool(np.all(np.isfinite(growth)))}


def time_paper_run(B, inputs, torch, stream, nsteps=2000):
    """The whole paper-scale run as one call: 32^3 from a = 1/51 to a = 1 in
    2000 KDK steps (FP32 compensated forces, FP64 a(t)), 64 tracers recorded
    every step, then their velocity energy spectra and the diagnostics."""
    ic = inputs.grid32()
    tau = inputs.lcdm_tau(nsteps)
    sim = B.Simulation(ic.m, ic.eps, LCDM, inputs.A_START, prec=B.FP32_COMP, scheme=B.KDK,
                       stream=stream.cuda_stream)
    try:
        sim.set_state(ic.x, ic.v)
        sim.record_tracers(inputs.tracers(ic.N, 64, 7), nsteps)
        sim.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        t0 = time.perf_counter()
        ev[0].record(stream)
        sim.step(tau, nsteps)
        ev[1].record(stream)
        spec = sim.tracer_spectrum(tau, "hann")
        ev[2].record(stream)
        diag = sim.diagnostics()
        wall = time.perf_counter() - t0
        # the first spectrum call also loads its kernels; a repeat shows the steady cost
        sim.synchronize()
        ev[3].record(stream)
        sim.tracer_spectrum(tau, "hann")
        ev[4].record(stream)
        stream.synchronize()
        # a repeat of the diagnostics (O(N^2) potential energy, moments)
        ev[5].record(stream)
        sim.diagnostics()
        ev[6].record(stream)
        stream.synchronize()
        _, _, t, a = sim.state()
    finally:
        sim.close()
    steps_ms = ev[0].elapsed_time(ev[1])
    return {"N": ic.N, "steps": nsteps, "a_final": a, "t_final": t,
            "steps_ms": steps_ms, "steps_per_s": nsteps / (steps_ms * 1e-3),
            "spectrum_ms": ev[3].elapsed_time(ev[4]), "spectrum_first_call_ms": ev[1].elapsed_time(ev[2]),
            "spectrum_shape": list(spec.shape), "diagnostics_ms": ev[5].elapsed_time(ev[6]),
            "wall_s_with_readback": wall, "finite": bool(np.isfinite(diag["K"])),
            "what": "one colatus_step call of 2000 steps, then colatus_tracer_spectrum and "
                    "colatus_diagnostics; the paper's only run was this size on a GTX680, "
                    "with no time reported"}


def time_schemes(B, inputs, torch, stream, nsteps=50):
    """The step variants on the 32^3 workload, FP32 compensated force, one
    colatus_step call of nsteps after two warm-up steps (L2 not flushed; the
    state is 1 MB): the paper's DKD (Eqs. 3-5), the drag KDK, the canonical
    (symplectic) KDK of Sec. II, and the drag KDK with the Eq. 6 deformation
    term.  All run the same force kernel; the variants differ in O(N) epilogue
    work and in the FP64 schedule."""
    ic = inputs.grid32()
    tau = inputs.lcdm_tau(2000)
    out = {}
    for name, scheme, defo in (("dkd", B.DKD, False), ("kdk", B.KDK, False),
                               ("kdk_canonical", B.KDK_CANONICAL, False),
                               ("kdk_deformation", B.KDK, True)):
        sim = B.Simulation(ic.m, ic.eps, LCDM, inputs.A_START, prec=B.FP32_COMP, scheme=scheme,
                           stream=stream.cuda_stream)
        try:
            sim.set_state(ic.x, ic.v)
            if defo:
                sim.set_deformation(0.01 * float(np.sum(ic.m)), np.array([0.5, 0.5, 0.5]))
            sim.step(tau, 2)
            sim.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(tau, nsteps)
            e1.record(stream)
            torch.cuda.synchronize()
        finally:
            sim.close()
        ms = e0.elapsed_time(e1) / nsteps
        out[name] = {"ms_per_step": ms, "interactions_per_s": float(ic.N) * ic.N / (ms * 1e-3)}
    out["what"] = (f"{nsteps} steps of 32^3 per variant in one colatus_step call, FP32 compensated, "
                   "L2 not flushed")
    return out


def time_periodic(B, inputs, torch, stream, nsteps=10):
    """Periodic boundaries (Ewald summation) on the 32^3 workload, FP32
    compensated KDK: per step the real-space all-pairs kernel (minimum images),
    the k-space structure factors and long-range force, and the epilogue."""
    ic = inputs.grid32()
    tau = inputs.lcdm_tau(2000)
    sim = B.Simulation(ic.m, ic.eps, LCDM, inputs.A_START, prec=B.FP32_COMP, scheme=B.KDK,
                       stream=stream.cuda_stream)
    try:
        sim.set_state(ic.x, ic.v)
        sim.set_periodic(1.0)
        sim.step(tau, 2)
        sim.synchronize()
        sim.profile_forces(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(tau, nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        fms, n = sim.profile_read()
        sim.profile_forces(False)
        par = sim.periodic_params()
        # the force VJP under periodic boundaries (device buffers): the whole
        # call, and its real-space kernel alone
        w = torch.randn((ic.N, 3), device="cuda", dtype=torch.float32)
        gx, gm = torch.empty_like(w), torch.empty(ic.N, device="cuda", dtype=torch.float32)
        B.colatus_force_vjp(sim.h, w, gx, gm)          # loads the kernels (lazy loading)
        sim.synchronize()
        sim.profile_forces(True)
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        B.colatus_force_vjp(sim.h, w, gx, gm)
        e3.record(stream)
        torch.cuda.synchronize()
        vms, vn = sim.profile_read(vjp=True)
        sim.profile_forces(False)
        vjp_kind = sim.vjp_plan()["kind"]
    finally:
        sim.close()
    ms = e0.elapsed_time(e1) / nsteps
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    pairs = float(ic.N) * ic.N
    return {"N": ic.N, "box": 1.0, "alpha": par["alpha"], "nk": par["nk"], "k_vectors": par["nkv"],
            "ms_per_step": ms, "interactions_per_s": pairs / (ms * 1e-3),
            "real_space_ms_per_launch": fms / n,
            "real_space_interactions_per_sm_per_clk": pairs / (fms / n * 1e-3) / (nsm * 2.032e9),
            "vjp_call_ms": e2.elapsed_time(e3), "vjp_plan": vjp_kind,
            "vjp_real_space_ms": vms / max(1, vn),
            "vjp_real_space_interactions_per_sm_per_clk": pairs / (vms / max(1, vn) * 1e-3) /
            (nsm * 2.032e9),
            "what": "KDK step with periodic boundaries; real space = the minimum-image "
                    "all-pairs kernel alone (events around it); vjp = colatus_force_vjp on device "
                    "buffers (real space plus the reciprocal-space VJP)"}


def run_colatus(args, ws, rank, local):
    import torch
    from paper_1208_3444_b300 import binding as B
    from paper_1208_3444_b300 import inputs
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)      # the library and the events share it
    torch.cuda.set_stream(stream)
    props = torch.cuda.get_device_properties(dev)
    nsm = props.multi_processor_count

    ic = inputs.grid32()
    N = ic.N
    tau = inputs.lcdm_tau(2000)
    tr = inputs.tracers(N, 64, 7)
    K, W = args.steps, args.warmup
    sim = B.Simulation(ic.m, ic.eps, LCDM, inputs.A_START, prec=B.FP32_COMP, scheme=B.KDK,
                       stream=stream.cuda_stream)
    sim.set_state(ic.x, ic.v)
    sim.record_tracers(tr, K + W + 8)
    sim.step(tau, W)
    sim.synchronize()

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    launches0 = sim.stats()["launches"]
    plan = sim.force_plan()
    sim.profile_forces(True)
    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(K):
        flush.zero_()                       # L2 flush between timed steps (not timed)
        ev0[k].record(stream)
        sim.step(tau, 1)
        ev1[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(ws)
    clk = clocks.stop()
    step_ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    force_ms, nforce = sim.profile_read()
    sim.profile_forces(False)
    launches = sim.stats()["launches"] - launches0
    sim.synchronize()

    step_ms_max = max_over_ranks(ws, step_ms)
    value = aggregate_throughput(ws, K, float(N) * N, step_ms_max)

    # end to end through the C ABI with host buffers: the initial state from
    # pinned host memory, then per step the paper's host loop (Appendix A,
    # step 8): advance, then copy every position and velocity to the host.
    # The read-back is colatus_get_state_async (device snapshot, copy on a
    # second stream into pinned memory), so the copy of step k overlaps step
    # k+1; the last copy is waited for inside the timed region.
    Ke = min(K, 100)
    xh = torch.tensor(ic.x, dtype=torch.float32).pin_memory()
    vh = torch.tensor(ic.v, dtype=torch.float32).pin_memory()
    xo = [torch.empty((N, 3), dtype=torch.float32).pin_memory() for _ in range(4)]
    vo = [torch.empty((N, 3), dtype=torch.float32).pin_memory() for _ in range(4)]
    # the first asynchronous read-back creates the library's copy stream and
    # device snapshot slots (cudaMalloc, which synchronises the device): a
    # one-time setup, done before the timed region
    B.colatus_get_state_async(sim.h, xo[0], vo[0])
    B.colatus_wait_state(sim.h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.set_state(xh, vh)
    for k in range(Ke):
        sim.step(tau, 1)
        B.colatus_get_state_async(sim.h, xo[k % 4], vo[k % 4])
    B.colatus_wait_state(sim.h)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(ws, e2e_s)
    e2e = {"value": ws * Ke * float(N) * N / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(2 * N * 3 * 4 / Ke), "d2h_bytes_per_step": 2 * N * 3 * 4,
           "steps": Ke,
           "what": "per step: colatus_step + colatus_get_state_async of x and v into pinned host "
                   "memory (overlapping the next step); the initial colatus_set_state from pinned "
                   "host memory and the wait for the last copy are inside the timed region; one "
                   "untimed read-back before it creates the library's copy stream and slots"}
    sim.close()

    result = None
    force128 = None
    if not args.no_128:
        force128 = time_force_128(B, inputs, torch)
    adjoint = time_adjoint(B, inputs, torch, stream)
    ensemble = time_ensemble(B, inputs, torch, stream)
    tangent = time_tangent(B, inputs, torch, stream)
    periodic = time_periodic(B, inputs, torch, stream)
    schemes = time_schemes(B, inputs, torch, stream)
    paper_run = time_paper_run(B, inputs, torch, stream)
    pipes = B.colatus_probe_pipes()
    if rank == 0:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except (OSError, ValueError):
            pass
        f_mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
        fmax = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2032.0)
        achieved_int = float(N) * N * nforce / (force_ms * 1e-3)
        achieved = achieved_int * FLOPS_PER_INTERACTION / 1e12
        peak = nsm * FP32_FLOP_PER_CLK_PER_SM * f_mhz * 1e6 / 1e12
        traffic, same_shape, same_source = force_traffic(plan)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_note": ("dram__bytes_read.sum + dram__bytes_write.sum per launch of "
                                 f"{FORCE_KERNEL_TRAFFIC['template']} from one ncu capture; "
                                 f"launched kernel has the captured shape: {same_shape}; sources "
                                 f"unchanged since the capture: {same_source}; algorithmic HBM "
                                 "bytes: 524288 (positions read once)"),
                "kernel": ("force_sym_f32_kernel (FP32 compensated, every pair once, stream-K over "
                           "the tile pairs)" if plan.get("kind") == "force_sym_f32"
                           else "force_f32_kernel (FP32 compensated, stream-K)"),
                "launched_plan": plan,
                "interactions_per_s": achieved_int,
                "int_per_sm_per_clk": achieved_int / (nsm * f_mhz * 1e6),
                "peak_basis": f"{nsm} SMs x {FP32_FLOP_PER_CLK_PER_SM} FP32 flop/clk x "
                              f"{f_mhz:.0f} MHz (median sampled SM clock); 20 flop/interaction",
                "frac_at_max_clock": achieved / (nsm * FP32_FLOP_PER_CLK_PER_SM * fmax * 1e6 / 1e12),
                "ms_per_launch": force_ms / nforce,
                # the same rate against the FP32 pipe: lane-ops the launched
                # kernel's pair arithmetic needs per counted interaction (fewer
                # than the convention's 20 flops when every pair is evaluated
                # once, so frac may exceed 1 while the pipe stays below it)
                "fp32_lane_ops_per_interaction": pair_lane_ops(plan, N),
                "fp32_lane_op_frac": achieved_int / (nsm * f_mhz * 1e6) * pair_lane_ops(plan, N) / 128.0}
        if force128:
            a128 = force128["interactions_per_s"]
            force128["frac"] = a128 * FLOPS_PER_INTERACTION / 1e12 / peak
            ops128 = pair_lane_ops(force128["plan"], force128["N"])
            force128["fp32_lane_ops_per_interaction"] = ops128
            force128["fp32_lane_op_frac"] = a128 / (nsm * f_mhz * 1e6) * ops128 / 128.0
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
            "warmup": W, "ms_per_step": step_ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "grid32: N=32^3 perturbed grid, growing-mode velocities, "
                                   "eps=0.02 spacing, one KDK step (FP32 compensated force, FP64 "
                                   "a(t), Hubble drag, 64 tracers)",
                       "N": N, "prec": "fp32_comp", "scheme": "kdk", "tau": tau,
                       "l2": "flushed between timed steps (256 MiB write, outside the events)",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "steps_per_s": K / (step_ms_max * 1e-3),
            "wall_s_timed_region": wall,
            "roofline": roof,
            "force_128cubed": force128,
            "adjoint": adjoint,
            "ensemble": ensemble,
            "tangent": tangent,
            "periodic": periodic, "schemes": schemes,
            "paper_run": paper_run,
            "pipe_rates": {**pipes, "unit": "lane-ops (MUFU: results) per SM per clock",
                           "what": "colatus_probe_pipes: independent chains of FFMA, FFMA2 "
                                   "(f32x2), MUFU.RSQ"},
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
        if not args.no_cpu:
            result["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        # the headline figures again, last, so that a cut-off copy of the line keeps them
        result["headline"] = {
            "force_32cubed_frac": roof["frac"],
            "force_128cubed_frac": force128["frac"] if force128 else None,
            "force_128cubed_ms": force128["ms_per_launch"] if force128 else None,
            "force_128cubed_interactions_per_s": force128["interactions_per_s"] if force128 else None,
            "force_32cubed_fp32_lane_op_frac": roof["fp32_lane_op_frac"],
            "force_128cubed_fp32_lane_op_frac": force128["fp32_lane_op_frac"] if force128 else None,
            "adjoint_step_over_forward_step": adjoint["adjoint_step_over_forward_step"],
            "vjp_frac_of_lane_op_floor": adjoint["vjp_frac_of_lane_op_floor"],
            "ensemble_frac_of_fp32_roofline": ensemble["frac_of_fp32_roofline"],
            "periodic_real_space_int_per_sm_per_clk": periodic["real_space_interactions_per_sm_per_clk"],
            "e2e_over_value": e2e["value"] / value,
        }
    return result


def main():
    args = parse()
    if args.impl == "reference":
        # the oracle runs on rank 0's host cores only; other ranks exit without work
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        res = run_reference(args, ws, rank)
        if rank == 0 and res is not None:
            print(json.dumps(res), flush=True)
        return
    ws, rank, local = dist_setup()
    res = run_colatus(args, ws, rank, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
