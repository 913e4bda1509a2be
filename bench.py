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
import tempfile
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
    ap.add_argument("--traj", type=int, default=0,
                    help="small case: N trajectories (H = (N-1)//2) instead of the workload's")
    ap.add_argument("--newmark-steps", type=int, default=0,
                    help="small case: integrate only the first K Newmark steps of the period")
    ap.add_argument("--batch", action="store_true",
                    help="also time the 8-point shell batch (N = 32..64) as one graph against one by one")
    ap.add_argument("--predictor", default="mlp", choices=["secant", "mlp", "both"],
                    help="continuation predictor of --points (both: the two sweeps one after the other)")
    ap.add_argument("--points", type=int, default=-1,
                    help="also time K converged continuation points (chord corrector, GMRES outer solve); "
                         "default: 8 on one GPU, 0 under torchrun")
    ap.add_argument("--fp64-points", type=int, default=-1,
                    help="converged continuation points of the plain FP64 form timed for the points/s "
                         "comparison (default: 1 when --points runs)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the GEMM peak measurements")
    ap.add_argument("--solve", default="auto", choices=["auto", "simt", "tc"],
                    help="banded tangent-solve kernels (fse_set_tangent_solve)")
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
        # the raw samples are kept beside the run's other outputs (FSE_BENCH_OUT), else in /tmp
        out_dir = os.environ.get("FSE_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, "clocks_bench_%d.csv" % os.getpid())

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


def rank_omega(wl, rank):
    """Every rank solves its own continuation point (weak scaling, no exchange of
    trajectory data): w_1 of rank r is the workload's w_1 times 1 + 0.01 r."""
    return wl.omega1 * (1.0 + 0.01 * rank)


def max_over_ranks(ms, world, device):
    """Step time of the whole job: the slowest rank's (all-reduce MAX; the only collective)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (ms / 1e3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def csr_counts(m):
    """Nonzeros of the union pattern of M, D, K and of the K_t pattern of the nonlinear elements."""
    nnz = int(np.count_nonzero((m.M != 0) | (m.D != 0) | (m.K != 0)))
    kt = set()
    for e in range(m.n_nl):
        dofs = [int(x) for x in m.nl_dof[e] if x >= 0]
        for a in dofs:
            for b2 in dofs:
                kt.add((a, b2))
    return nnz, len(kt)


def step_work(m, N, band, ld, prec_bytes):
    """Algorithmic FP32 flops and HBM bytes per launch (all N trajectories, one Newmark step)
    of the three sensitivity kernels:
      rhs  Y = (A - K_t(q_k)) X_k + B V_k on the CSR patterns: 2 (2 nnz + nnz_kt) P flops,
           reads X, V and writes Y: 3 n P words;
      fwd  L Y' = Y (band b): 2 (n b - b (b + 1) / 2) P flops, reads Y and writes Y': 2 n P words;
      bwd  L^T X_{k+1} = Y' and V_{k+1} = 2/D (X_{k+1} - X_k) - V_k: the same flops + 3 n P,
           reads Y', X_k, V_k and writes X_{k+1}, V_{k+1}: 5 n P words.
    P = 2n + 1 tangent columns; the padding columns (P..ld) are not counted."""
    n, P, b = m.n, 2 * m.n + 1, band
    nnz, nnz_kt = csr_counts(m)
    tri = n * b - b * (b + 1) / 2
    w = prec_bytes
    return {
        "sens_rhs": (2.0 * (2 * nnz + nnz_kt) * P * N, 3.0 * n * P * w * N),
        "sens_fwd": (2.0 * tri * P * N, 2.0 * n * P * w * N),
        "sens_bwd": ((2.0 * tri + 3.0 * n) * P * N, 5.0 * n * P * w * N),
    }


def step_rates(work, traj_steps_per_s, N, hbm_gbs, fp64_tflops=None, bf16_tflops=None):
    """Whole-step rates of the tangent propagation from the measured throughput: the algorithmic
    bytes and flops of the three sensitivity kernels per Newmark step of all N trajectories
    (`step_work`), over the time of one such step, against the HBM peak and as multiples of the
    FP64 and BF16 tensor peaks (the tangent flops are FP32, so the FP64 ratio exceeds 1; the state
    step's FP64 work, the DFTs and the outer solves are not counted)."""
    t = N / traj_steps_per_s
    by = sum(v[1] for v in work.values())
    fl = sum(v[0] for v in work.values())
    gbs = by / t / 1e9
    tf = fl / t / 1e12
    return {"tangent_bytes_per_step": by, "hbm_gbs": gbs, "hbm_frac": gbs / hbm_gbs,
            "tangent_flops_per_step": fl, "tflops": tf,
            "vs_fp64_peak": tf / fp64_tflops if fp64_tflops else None,
            "vs_bf16_peak": tf / bf16_tflops if bf16_tflops else None}


def kernel_source_hash(source="fse_sens.cu"):
    """Hash of a kernel file's device code: the .cu file up to its host launchers, plus the device
    helpers of fse_common.cuh, with // comments and whitespace removed (a change in host code or
    in a comment leaves it unchanged, any change of the device code does not)."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2508_06302_gb300", "csrc")
    dev = open(os.path.join(csrc, source)).read().split("// launchers", 1)[0]
    dev += open(os.path.join(csrc, "fse_common.cuh")).read()
    code = re.sub(r"\s+", "", re.sub(r"//[^\n]*", "", dev))
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def recorded_traffic(kernel, workload_name, source="fse_sens.cu"):
    """DRAM bytes per launch recorded by an ncu capture in profiles/, with the hash of the
    kernel sources it was taken on; None when absent or when the sources changed since."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload_name))
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        if line.startswith("- ") and ": " in line:
            k, v = line[2:].split(": ", 1)
            rec[k.strip()] = v.strip().strip("`")
    h = kernel_source_hash(source)
    if rec.get("sources_sha256_16") != h:
        return None
    try:
        return float(rec["dram_bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


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
    threads = blas_threads()
    return {"value": done / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "host_cores": len(os.sched_getaffinity(0)),
            "sample": "%d traj-steps (with sensitivities) of one trajectory of %s in %.1f s: the NumPy FP64 "
                      "oracle as it stands, dense np.linalg.solve per Newton iteration and per tangent solve "
                      "(no band, no parallelism over trajectories), BLAS threads %d"
                      % (done, wl.name, el, threads)}


def blas_threads():
    """Threads of the BLAS the oracle's dense solves run on (threadpoolctl when present, else the
    usual environment settings, else every host core: OpenBLAS's default)."""
    try:
        from threadpoolctl import threadpool_info
        n = [int(d.get("num_threads", 0)) for d in threadpool_info() if d.get("user_api") == "blas"]
        if n and max(n) > 0:
            return max(n)
    except Exception:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        v = os.environ.get(var)
        if v and v.isdigit() and int(v) > 0:
            return int(v)
    return len(os.sched_getaffinity(0))


def gemm_peaks(torch):
    """Measured dense-GEMM peaks of this GPU through cuBLAS (torch.matmul), best of several
    launches timed with CUDA events: FP32 with TF32 off (the SIMT FMA pipes), TF32 tensor cores,
    FP64 (DGEMM).  These are the denominators of the FP32 / TF32 / FP64 roofline fractions."""
    prev = torch.backends.cuda.matmul.allow_tf32
    out = {}
    try:
        for key, dtype, n, tf32, reps in (("fp32_simt_tflops", torch.float32, 8192, False, 5),
                                         ("tf32_tflops", torch.float32, 8192, True, 8),
                                         ("fp64_tflops", torch.float64, 4096, False, 3)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            g = torch.Generator(device="cuda")
            g.manual_seed(0)
            a = torch.randn(n, n, dtype=dtype, device="cuda", generator=g)
            b = torch.randn(n, n, dtype=dtype, device="cuda", generator=g)
            c = torch.empty(n, n, dtype=dtype, device="cuda")
            for _ in range(2):
                torch.matmul(a, b, out=c)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[key] = 2.0 * n ** 3 / (best / 1e3) / 1e12
            del a, b, c
        out["how"] = ("torch.matmul square GEMMs (FP32 8192^3 TF32 off and on, FP64 4096^3), 2 n^3 flops, "
                      "best of 5/8/3 CUDA-event-timed launches")
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def batch_points(fse, device):
    """The 8 continuation points of uneven trajectory count (N = 32..64, H = (N-1)//2,
    w_1 = w_n1 {0.95..1.3}) evaluated with their Jacobians as one captured CUDA graph,
    against the same evaluations one context at a time (the graph is captured by an
    untimed first call)."""
    from paper_2508_06302_gb300 import inputs as I
    wls = I.shell_batch_points()
    ctxs = [fse.Context.from_workload(w, precision="mixed_fp32", device=device) for w in wls]
    Zs = [initial_coeffs(w) for w in wls]
    om = [w.omega1 for w in wls]
    b = fse.Batch(ctxs, use_graph=True)
    b.residual_jacobian(Zs, om, True)
    t0 = time.perf_counter()
    Rs, st, rc = b.residual_jacobian(Zs, om, True)
    t_graph = time.perf_counter() - t0
    t0 = time.perf_counter()
    for c, z, w in zip(ctxs, Zs, om):
        c.residual_jacobian(z, w, True)
    t_seq = time.perf_counter() - t0
    ts = sum(w.N * w.S1 for w in wls)
    b.close()
    for c in ctxs:
        c.close()
    return {"points": len(wls), "trajectories": sum(w.N for w in wls), "status": [int(x) for x in st],
            "graph_s": t_graph, "one_by_one_s": t_seq, "traj_steps_per_s_graph": ts / t_graph,
            "traj_steps_per_s_one_by_one": ts / t_seq, "speedup": t_seq / t_graph}


def continuation_points(fse, ctx, wl, K, predictor="secant", device=0):
    """K + 1 points of the w_1 sweep from 0.90 w_n1 in steps of 0.002 w_n1: the first converged
    from the discrete linear response (not counted), then K points with the secant predictor, or
    the secant corrected by the BF16 network trained online on the secant's errors (64 POD modes,
    warm-up 4 points), and the chord corrector (one Jacobian per point, GMRES on the structured
    products for the outer solve), each accepted at ||R|| <= 1e-10 ||Z|| (FP64 residual)."""
    import dataclasses
    from paper_2508_06302_gb300 import inputs as I
    w_n1 = wl.model.omega_n1
    omegas = w_n1 * (0.90 + 0.002 * np.arange(K + 1))
    Z0 = initial_coeffs(dataclasses.replace(wl, omega1=float(omegas[0])))
    ctx.set_steps(0)
    ctx.profile(False)
    net = None
    kw = {}
    if predictor == "mlp":
        net = fse.Mlp(3, 256, 64, max_batch=max(64, K + 1), device=device)
        net.set_params(I.mlp_init(3, 256, 64, seed=0))
        kw = dict(predictor="mlp", mlp=net, warmup=4, pod_modes=64, pod_every=1, train_steps=300, lr=2e-3)
    Z, pts, rc = fse.fse_continue(ctx, omegas, Z0, rel_tol=1e-10, max_newton=40, chord=True, **kw)
    if net is not None:
        net.close()
    timed = pts[1:]
    tot_ms = sum(p["ms"] for p in timed)
    lin = ctx.linear_stats()
    continuation_points.last = (omegas, Z, pts)
    return {"points": K, "predictor": predictor, "points_per_s": K / (tot_ms / 1e3) if tot_ms > 0 else None,
            "ms_per_point": [round(p["ms"], 1) for p in timed],
            "newton_iters": [p["newton_iters"] for p in timed],
            "pred_err": [p["pred_err"] for p in timed],
            "learned_used": [p["predictor"] == fse.FSE_PRED_MLP for p in timed],
            "jacobian_evals_per_point": 1,
            "residual_evals": [p["evals"] - 1 for p in timed],
            "rel_res": [p["res"] / p["znorm"] for p in timed],
            "status": [p["status"] for p in timed], "rc": rc,
            "first_point": {"ms": round(pts[0]["ms"], 1), "newton_iters": pts[0]["newton_iters"],
                            "status": pts[0]["status"]},
            "last_gmres": {"iters": lin[0], "rel_res": lin[1]},
            "omega1_over_wn1": [round(float(w / w_n1), 4) for w in omegas]}


def fp64_points(fse, wl, omegas, Zconv, pts_mixed, K, device):
    """The plain FP64 form (FP64 sensitivities, secant predictor, the same chord corrector and
    GMRES outer solve) on K converged points of the same sweep: point j (j = 1..K) is corrected
    from the mixed form's converged point j - 1, the prediction the mixed sweep also makes at
    j = 1.  Its accepted tori are compared with the mixed form's (both accepted at
    ||R|| <= 1e-10 ||Z||)."""
    c64 = fse.Context.from_workload(wl, precision="fp64", device=device)
    ms, its, diffs, sts = [], [], [], []
    for j in range(1, K + 1):
        Z, pts, rc = fse.fse_continue(c64, omegas[j:j + 1], Zconv[j - 1], rel_tol=1e-10, max_newton=40,
                                      chord=True)
        ms.append(pts[0]["ms"])
        its.append(pts[0]["newton_iters"])
        sts.append(pts[0]["status"])
        diffs.append(float(np.linalg.norm(Z[0] - Zconv[j]) / np.linalg.norm(Zconv[j])))
    c64.close()
    tot = sum(ms)
    return {"points": K, "predictor": "previous point (the mixed sweep's point-1 prediction)",
            "points_per_s": K / (tot / 1e3), "ms_per_point": [round(x, 1) for x in ms], "newton_iters": its,
            "status": sts, "rel_diff_vs_mixed_torus": diffs,
            "mixed_same_start_ms": round(pts_mixed[1]["ms"], 1)}


def half_bandwidth(model):
    """Half-bandwidth of the union pattern of M, D, K and the nonlinear elements' dof spans."""
    i, j = np.nonzero((model.M != 0) | (model.D != 0) | (model.K != 0))
    b = int(np.max(np.abs(i - j))) if i.size else 0
    for dofs in model.nl_dof:
        d = [int(x) for x in dofs if x >= 0]
        if len(d) > 1:
            b = max(b, max(d) - min(d))
    return b


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
                                            "H": wl.H, "S1": wl.S1, "band": half_bandwidth(wl.model),
                                            "precision": "fp64 (oracle)"},
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
    if args.traj > 0:
        import dataclasses
        wl = dataclasses.replace(wl, S=[args.traj], H=[(args.traj - 1) // 2],
                                 name=wl.name + "_N%d" % args.traj)
    m = wl.model
    # every rank runs its own continuation point (weak scaling, no exchange)
    w1 = rank_omega(wl, rank)
    ctx = fse.Context.from_workload(wl, precision=args.precision, device=local)
    if args.solve != "auto":
        ctx.set_tangent_solve(args.solve)
    ctx.profile(True)
    n_newmark = wl.S1
    if 0 < args.newmark_steps < wl.S1:
        n_newmark = args.newmark_steps
        ctx.set_steps(n_newmark)
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
    phase = np.zeros(6)
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
        ms = max_over_ranks(ms, world, "cuda")
        torch.distributed.barrier()
    traj_steps = wl.N * n_newmark
    value = job_value(traj_steps, world, ms)
    phase /= args.steps                 # per step; phase[5] is the mean refactor count

    # end-to-end through the host-pointer API (H2D of Z(0), D2H of R inside the timed region)
    Zh = initial_coeffs(wl)
    t0 = time.perf_counter()
    n_e2e = max(1, min(3, args.steps // 2))
    for _ in range(n_e2e):
        Rh, st_h, it_h, rc_h = ctx.residual_jacobian(Zh, w1, True)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / n_e2e

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

    peaks_gemm = None if args.no_peaks else gemm_peaks(torch)
    peaks, src = measured_peaks()
    # per-kernel rooflines of the sensitivity kernels (FP32 / FP64 SIMT arithmetic or HBM,
    # whichever bounds the kernel) from their event-timed average launch duration on the
    # launching stream
    names = ["state", "sens_rhs", "sens_fwd", "sens_bwd"]
    b = ctx.band
    n, N = m.n, wl.N
    wb = 4 if args.precision == "mixed_fp32" else 8
    work = step_work(m, N, b, 0, wb)
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    lanes = 128 if wb == 4 else 2            # FP32 / FP64 SIMT lanes per SM (FP64: 1/64 of FP32)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    alu_derived = n_sm * lanes * 2 * sm_mhz * 1e6 / 1e12
    gkey = "fp32_simt_tflops" if wb == 4 else "fp64_tflops"
    alu_peak = peaks_gemm[gkey] if peaks_gemm else alu_derived
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # the banded solves run on the TF32 tensor cores (FP32 tangents, b <= 96): three TF32 products
    # per FP32-accurate product, so their compute roof is a third of the measured TF32 GEMM rate
    tc = wb == 4 and b <= 96 and args.solve == "tc"
    tf32 = (peaks_gemm or {}).get("tf32_tflops") or 0.5 * peaks.get("bf16_tflops", 1900.0)
    kernels = {}
    for k_i, kname in enumerate(names):
        if kname not in work:
            continue
        avg_ms = phase[1 + k_i] / n_newmark
        if avg_ms <= 0:
            continue
        fl, by = work[kname]
        on_tc = tc and kname in ("sens_fwd", "sens_bwd")
        cpeak = tf32 / 3.0 if on_tc else alu_peak
        t_alu = fl / (cpeak * 1e12)
        t_hbm = by / (hbm_peak * 1e9)
        if t_alu >= t_hbm:
            ach = fl / (avg_ms / 1e3) / 1e12
            kernels[kname] = {"bound": "tensor" if on_tc else "alu", "achieved": ach, "peak": cpeak,
                              "unit": "TFLOP/s", "frac": ach / cpeak, "avg_launch_ms": avg_ms,
                              "algorithmic_flops": fl, "algorithmic_bytes": by}
        else:
            ach = by / (avg_ms / 1e3) / 1e9
            kernels[kname] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                              "frac": ach / hbm_peak, "avg_launch_ms": avg_ms,
                              "algorithmic_flops": fl, "algorithmic_bytes": by}
        kernels[kname]["kernel"] = {"state": "k_state", "sens_rhs": "k_sens_rhs",
                                    "sens_fwd": "k_tc_records + k_tc_solve<fwd>" if on_tc else "k_trsm8<fwd>",
                                    "sens_bwd": "k_tc_solve<bwd>" if on_tc else "k_trsm8<bwd>"}[kname]
    roof = None
    if kernels:
        kname = max(kernels, key=lambda k: kernels[k]["avg_launch_ms"])
        kk = kernels[kname]
        on_tc = tc and kname in ("sens_fwd", "sens_bwd")
        tname = ("k_tc_solve_" + kname[5:]) if on_tc else ("k_" + kname)
        if kk["bound"] == "hbm":
            psrc = "%s of %s (HBM copy)" % (hbm_peak, src)
        elif kk["bound"] == "tensor":
            psrc = ("measured cuBLAS TF32 GEMM / 3 (three TF32 products per FP32-accurate product)" if peaks_gemm
                    else "half the measured BF16 GEMM rate / 3")
        elif peaks_gemm:
            psrc = "measured cuBLAS %s GEMM (%s)" % ("FP32 TF32-off" if wb == 4 else "FP64", gkey)
        else:
            psrc = "%d SMs x %d lanes x 2 flop x median SM clock %.0f MHz (derived)" % (n_sm, lanes, sm_mhz)
        roof = {"kernel": kname, "kernel_name": kk["kernel"], "bound": kk["bound"], "achieved": kk["achieved"],
                "peak": kk["peak"], "unit": kk["unit"], "frac": kk["frac"],
                "traffic": recorded_traffic(tname, wl.name, "fse_tc.cu" if on_tc else "fse_sens.cu"),
                "peak_source": psrc}
    batch = None
    if args.batch:
        try:
            batch = batch_points(fse, local)
        except Exception as exc:
            batch = {"error": "%s: %s" % (type(exc).__name__, exc)}
    cont = None
    n_points = args.points if args.points >= 0 else (8 if world == 1 else 0)
    if n_points > 0:
        cont = {}
        # a sweep that fails is reported in the line; the timed evaluation above stands
        try:
            for p in (["secant", "mlp"] if args.predictor == "both" else [args.predictor]):
                cont[p] = continuation_points(fse, ctx, wl, n_points, p, local)
            omegas, Zc, pts_c = continuation_points.last
            k64 = args.fp64_points if args.fp64_points >= 0 else 1
            if k64 > 0:
                cont["fp64_plain"] = fp64_points(fse, wl, omegas, Zc, pts_c, min(k64, n_points), local)
                best = max(v["points_per_s"] or 0.0 for k, v in cont.items() if k != "fp64_plain")
                cont["vs_fp64_plain"] = best / cont["fp64_plain"]["points_per_s"]
        except Exception as exc:
            cont["error"] = "%s: %s" % (type(exc).__name__, exc)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl, args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 state / f32 sensitivities", "data": "synthetic",
        "config": {"workload": wl.name, "n": n, "N": N, "H": wl.H, "S1": wl.S1, "band": b,
                   "newmark_steps_timed": n_newmark,
                   "precision": args.precision, "l2": "working set >> L2 (no flush needed)"},
        "status": int(rc), "newton_iters_per_step": float(np.mean(its)) / n_newmark,
        "phase_ms": {nm: float(v) for nm, v in zip(["total"] + names, phase[:5])},
        "refactors_per_traj_step": float(phase[5]),
        "kernels": kernels,
        "e2e": {"value": traj_steps / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": nu * 8,
                "d2h_bytes_per_step": nu * 8 + 8 * N},
        "fp64_plain": fp64,
        "speedup_vs_fp64_plain": (value / fp64["value"]) if fp64 else None,
        # per evaluation: i-DFT, split, initial state, tangent init, S1 x (state step + the three
        # sensitivity kernels), join, DFT + residual
        # (+1 per step: the factor records of the tensor-core solves)
        "gpu_launches": args.steps * ((5 if tc else 4) * n_newmark + 6),
        "roofline": roof,
        # per GPU (each rank integrates its own N trajectories)
        "step_rates": step_rates(work, value / world, N, hbm_peak, (peaks_gemm or {}).get("fp64_tflops"),
                                 peaks.get("bf16_tflops")),
        "clocks": clk, "cpu_baseline": cpu, "peaks_source": src,
        "peaks_measured": peaks_gemm,
        "alu_peak_derived_tflops": alu_derived,
    }
    if cont is not None:
        line["continuation"] = cont
    if batch is not None:
        line["batch"] = batch
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
