"""Benchmark of the FSE-Shooting hot path on GB300.

One step = one full evaluation of the shooting residual and its Jacobian
(Eq. 16, Eq. 22): i-DFT of Z(0), Newmark + per-step Newton + sensitivity
propagation of all N trajectories over one period, DFT + rotation.  Workload:
the 1872-dof flat clamped shell, d = 2, N = 64 trajectories (H = 31),
S1 = 1000 Newmark steps, FP64 state with FP32 sensitivities.  Inputs are
seeded synthetic (no dataset); the per-step working set (tangent arrays of
1.8 GB each) is far larger than L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "traj-steps/s"
UNIT = "traj-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fse", choices=["fse", "reference"])
    ap.add_argument("--workload", default="shell1872")
    ap.add_argument("--precision", default="mixed_fp32")
    ap.add_argument("--fp64-steps", type=int, default=10,
                    help="Newmark steps of the plain FP64 form timed for the comparison line")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def workload(name):
    from paper_2508_06302_gb300 import inputs as I
    if name == "shell1872":
        return I.workload_shell1872()
    if name == "beam18":
        return I.workload_beam18()
    if name == "vkbeam447":
        return I.workload_vkbeam447()
    if name == "plate243":
        return I.workload_plate243()
    raise SystemExit("unknown workload " + name)


def initial_coeffs(wl):
    """Deterministic start: the discrete linear response (f_nl dropped), as a Newton start."""
    import math
    m = wl.model
    n = m.n
    U = wl.U_tilde
    Dl = 2 * math.pi / wl.S1
    w1 = wl.omega1
    C = np.zeros((2 * n, U))
    comps = [(1.0, m.F[0], None)]
    if m.F.shape[0] > 1 and wl.d == 2:
        comps.append((wl.rho[0], m.F[1], 1))
    for lam, F, col in comps:
        s = 2j / Dl * math.tan(lam * Dl / 2)
        Q = np.linalg.solve(m.K + w1 * s * m.D + w1 ** 2 * s * s * m.M, F)
        if col is None:
            C[:n, 0], C[n:, 0] = Q.real, (s * Q).real
        else:
            C[:n, 1], C[n:, 1] = Q.real, (s * Q).real
            C[:n, 2], C[n:, 2] = -Q.imag, -(s * Q).imag
    return C.reshape(-1)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(mx)
        out["reasons"] = sorted(reasons)
        return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def band_nnz(A):
    return int(np.count_nonzero(A))


def cpu_baseline(wl, seconds):
    """The CPU oracle, as it stands, on a bounded sample: trajectory-steps with sensitivities."""
    from oracle import fse_oracle as O
    m = wl.model
    prob = O.FSEProblem(m, wl.S, wl.H, wl.S1, wl.rho)
    Z = initial_coeffs(wl)
    zb = O.idft(prob, Z)
    done = 0
    t0 = time.perf_counter()
    steps = 1
    while True:
        O.integrate_trajectory(m, wl.omega1, prob.rho, prob.T[:, 0], zb[0, :m.n], zb[0, m.n:], wl.S1,
                               tol=wl.newton_tol, maxit=wl.newton_maxit, sens=True, n_steps=steps)
        done += steps
        el = time.perf_counter() - t0
        if el >= seconds or done >= 200:
            break
        steps = max(1, min(20, int(steps * 2)))
    return {"value": done / el, "unit": UNIT, "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": "%d traj-steps (with sensitivities) of one trajectory of %s in %.1f s"
                      % (done, wl.name, el)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args.workload)
    secs = max(3.0, args.cpu_seconds / max(1, args.steps))
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(wl, 1.0)
    t0 = time.perf_counter()
    samples = []
    for _ in range(args.steps):
        cb = cpu_baseline(wl, secs)
        vals.append(cb["value"])
        samples.append(cb["sample"])
    el = time.perf_counter() - t0
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "n": wl.model.n, "N": wl.N,
                                            "H": wl.H, "S1": wl.S1},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": len(os.sched_getaffinity(0)),
                             "kind": "oracle", "sample": samples[0]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2508_06302_gb300 import fse
    wl = workload(args.workload)
    m = wl.model
    # every rank runs its own continuation point (weak scaling, no exchange)
    w1 = wl.omega1 * (1.0 + 0.01 * rank)
    ctx = fse.Context.from_workload(wl, precision=args.precision, device=local)
    ctx.profile(True)
    nu = ctx.n_unknowns
    Z = torch.tensor(initial_coeffs(wl), dtype=torch.float64, device="cuda")
    R = torch.zeros(nu, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    def step():
        ctx.residual_jacobian_dev(Z.data_ptr(), w1, R.data_ptr(), True, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    rc, st, its = ctx.status()
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    phase = np.zeros(5)
    e0.record()
    for _ in range(args.steps):
        step()
        ctx.status()                    # waits; accumulates the per-kernel event timings
        phase += ctx.timings()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    traj_steps = wl.N * wl.S1
    value = traj_steps * world / (ms / 1e3)
    phase /= args.steps

    # end-to-end through the host-pointer API (H2D of Z(0), D2H of R inside the timed region)
    Zh = initial_coeffs(wl)
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps // 2)):
        Rh, st_h, it_h, rc_h = ctx.residual_jacobian(Zh, w1, True)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / max(1, args.steps // 2)

    # plain FP64 form of the same workload, timed on its first --fp64-steps Newmark steps
    fp64 = None
    if args.fp64_steps > 0:
        c64_short = fse.Context.from_workload(wl, precision="fp64", device=local)
        c64_short.set_steps(args.fp64_steps)
        Rd = torch.zeros(nu, dtype=torch.float64, device="cuda")
        c64_short.residual_jacobian_dev(Z.data_ptr(), w1, Rd.data_ptr(), True, stream)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        c64_short.residual_jacobian_dev(Z.data_ptr(), w1, Rd.data_ptr(), True, stream)
        f1.record()
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        fp64 = {"value": wl.N * args.fp64_steps / (ms64 / 1e3), "unit": UNIT,
                "sample": "%d of %d Newmark steps, all %d trajectories" % (args.fp64_steps, wl.S1, wl.N)}
        c64_short.close()

    peaks, src = measured_peaks()
    # dominant kernel and its roofline (FP32 SIMT arithmetic: alu bound)
    names = ["state", "sens_rhs", "sens_fwd", "sens_bwd"]
    k = int(np.argmax(phase[1:5]))
    nnzMD = band_nnz(m.M) + band_nnz(m.D)
    b = ctx.band
    n, P, N = m.n, 2 * m.n + 1, wl.N
    # algorithmic flops per step (one launch) of each sensitivity kernel
    flops = {"sens_rhs": 2.0 * nnzMD * P * N,
             "sens_fwd": 2.0 * (n * b - b * (b + 1) / 2) * P * N,
             "sens_bwd": 2.0 * (n * b - b * (b + 1) / 2) * P * N + 6.0 * n * P * N}
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12        # TFLOP/s of the FP32 SIMT pipes
    roof = None
    kname = names[k]
    if kname in flops:
        avg_ms = phase[1 + k] / wl.S1
        ach = flops[kname] / (avg_ms / 1e3) / 1e12
        roof = {"kernel": kname, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": None,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x median SM clock %.0f MHz" % sm_mhz}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl, args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 state / f32 sensitivities", "data": "synthetic",
        "config": {"workload": wl.name, "n": n, "N": N, "H": wl.H, "S1": wl.S1, "band": b,
                   "precision": args.precision, "l2": "working set >> L2 (no flush needed)"},
        "status": int(rc), "newton_iters_per_step": float(np.mean(its)) / wl.S1,
        "phase_ms": {nm: float(v) for nm, v in zip(["total"] + names, phase)},
        "e2e": {"value": traj_steps / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": nu * 8,
                "d2h_bytes_per_step": nu * 8 + 8 * N},
        "fp64_plain": fp64,
        "speedup_vs_fp64_plain": (value / fp64["value"]) if fp64 else None,
        "gpu_launches": 3 + wl.S1 * 4 + 4,
        "roofline": roof, "clocks": clk, "cpu_baseline": cpu, "peaks_source": src,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
