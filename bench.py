"""Benchmark: V-ASMG-PCG MDOF*iter/s to 1e-6 relative residual on GB300.

Headline workload (the largest single-GPU configuration): 3D linear
elasticity on a 128^3 vertex grid graded toward one corner (spacing ratio 16
per axis), 6 Kuhn tetrahedra per hex (6,291,456 dofs, 6,242,304 free), E = 1,
nu = 0.45, face x = 0 clamped, body force (0,0,-1); BF16 operator values in the
smoother, FP32 transfers and coarse operators, FP64 outer CG and coarsest
Cholesky.  One step = one full solve (every row of the hot path: FP64 SpMV +
CG updates + V-cycle with multicolour block GS, residual, restriction,
coarsest Cholesky solve, prolongation) from U0 = 0 to ||r||/||F|| < 1e-6.
The plain FP64 path on the same mesh is timed beside it, and so are the
other configurations (2D 64^2 FP64; 2D 1024^2 1:100 checkerboard, FP32
V-cycle and FP64; 3D 64^3 FP32 V-cycle), each with iterations and ms per solve.

value = sum(n_free * iterations) / device time / 1e6, inputs resident in HBM.
e2e   = the same through vasmg_solve with pinned host F and U (H2D + D2H in
        the timed region).
The operators (1.3 GB of level-0 FP64 blocks alone) exceed the 129 MB L2, so
no explicit flush is needed between timed steps.

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload: the same recipe at 32^3 vertices.
"""
from __future__ import annotations

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

WORKLOAD = "cube128_graded"
# V-cycle precision of each workload's configuration
DEFAULT_PRECISION = {"cube128_graded": "bf16", "cube64": "fp32", "square1024_checker": "fp32", "square64": "fp64"}
TAIL_NV = 20000         # levels this small run inside the single cluster tail launch
# CPU sample: the same recipe at this many vertices per side (a full oracle
# solve takes about 10 s on one core)
SAMPLE_N = {"cube128_graded": 32, "cube64": 32, "square1024_checker": 192, "square64": 64}
# DRAM bytes (read + write) of one launch from an ncu capture of the current
# kernel (profiles/); absent when the kernel changed after the capture.  The
# 128^3 entry is a one-pass capture (dram__bytes_read.sum + write.sum) of the
# full-size launch of the staged level-1 backward sweep: 2896.2 + 9.9 MB
# against 2291.9 MB algorithmic (the staged copy's padding slots and the
# gathers that miss L2).
TRAFFIC = {
    ("cube128_graded", "bwd_sweep_l1"): 2906166784.0,
}
TOL = 1e-6


def levels_vertices(s, l):
    from paper_2505_09064_gb300 import vasmg

    return vasmg.vasmg_level_info(s.h, l)[0]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "bf16"],
                    help="V-cycle precision (default: the workload's configuration)")
    ap.add_argument("--no-others", action="store_true", help="skip the other workloads' lines")
    ap.add_argument("--fp64-peak", action="store_true", help="only measure the FP64 FMA rate and print it")
    ap.add_argument("--side", type=int, default=0,
                    help="run the workload's recipe at this many vertices per side (profiling small cases)")
    ap.add_argument("--profile-kernel", default="",
                    help="KIND:LEVEL (KIND in spmv64, sweep, fwd_sweep, residual, restrict, prolong, tail): set "
                         "up the workload, then launch that kernel once between cudaProfilerStart/Stop (for "
                         "ncu --profile-from-start off) and print its CUDA-event time")
    ap.add_argument("--profile-k", type=int, default=1,
                    help="with --profile-kernel: launch the kernel with this many right-hand sides (2, 4 or 8; "
                         "vasmg_time_kernel_multi, FP32-vector precisions)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="lanes per row by rule (setup then launches no timing runs; for launch-indexed profiles)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every kernel from the host instead of one CUDA graph per solve")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--solve-only", action="store_true",
                    help="time the solves only (no per-kernel roofline timing, e2e, FP64 path or CPU "
                         "baseline); used for profiler launch lists")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = DEFAULT_PRECISION.get(args.workload, "fp32")
    return args


def reduce_over_ranks(ms: float, work: float, device=None):
    """Replicas: the job's time is the slowest rank's, its work the sum of all
    ranks' work.  Without an initialised process group, the local values."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return ms, work
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def sample_problem(workload: str, n: int):
    """The workload's recipe (mesh, material, boundary conditions, load) at n
    vertices per side."""
    from paper_2505_09064_gb300 import meshgen

    cfg = dict(meshgen.WORKLOADS[workload])
    return meshgen.make_problem(None, dim=cfg["dim"], n=n, jitter=cfg["jitter"], seed=cfg["seed"], E=cfg["E"],
                                nu=cfg["nu"], checker=cfg["checker"], graded=cfg["graded"])


def cpu_oracle_run(workload: str, n: int, steps: int, threads: int = 1):
    """Time the CPU oracle's solve on the workload's recipe at n vertices per
    side.  threads > 1 runs the oracle's OpenMP build (same bits, independent
    row loops on that many threads).  Returns (values, free dofs, threads used)
    with values = [(MDOF*iter/s, iterations, seconds)] per solve."""
    import oracle

    prob = sample_problem(workload, n)
    o = oracle.Oracle(prob, threads=threads)
    F = o.assemble_load(prob["body_force"])
    nfree = F.size - prob["dirichlet_dofs"].size
    vals = []
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        _, it, rr, st, _ = o.solve(F, tol=TOL)
        dt = time.perf_counter() - t0
        vals.append((nfree * it / dt / 1e6, it, dt))
    return vals, nfree, o.threads


def serving_requests(n_req: int, seed: int = 5):
    """The serving workload: mixed 2D/3D jittered meshes, dofs log-uniform in
    [5k, 500k], E ~ U[1,100], nu ~ U[0.2,0.45], 1-8 right-hand sides, each the
    load of a constant body force f ~ U[-1,1]^d."""
    from paper_2505_09064_gb300 import meshgen

    rs = meshgen.Stream(seed)
    out = []
    for i in range(n_req):
        u = rs.uniform(6)
        dim = 2 if u[0] < 0.5 else 3
        dofs = float(np.exp(np.log(5e3) + u[1] * (np.log(5e5) - np.log(5e3))))
        n = max(4, int(round((dofs / dim) ** (1.0 / dim))))
        E = 1.0 + 99.0 * u[2]
        nu = 0.2 + 0.25 * u[3]
        k = 1 + min(7, int(u[4] * 8))
        prob = meshgen.make_problem(None, dim=dim, n=n, jitter=0.2 if dim == 2 else 0.15, seed=seed * 1000 + i,
                                    E=E, nu=nu)
        forces = rs.uniform(k * dim, -1.0, 1.0).reshape(k, dim)
        out.append((prob, forces))
    return out


def serving_run(stream, n_req: int = 32):
    """Continuous-batching server on the serving workload: single-stream
    capacity, Poisson arrivals at 0.5/0.8/0.95 of it, and the plain FP64
    one-solve-at-a-time path on the same requests.  Each request's slot
    solves its right-hand sides together (vasmg_solve_multi); the batched
    executor (one launch per level and phase across requests) is run on the
    same arrivals beside it."""
    from paper_2505_09064_gb300 import meshgen, vasmg

    reqs = serving_requests(n_req)
    # right-hand sides assembled by the library (outside every timed region)
    loads = []
    for prob, forces in reqs:
        s = vasmg.Solver(prob, precision="fp64", stream=stream)
        n = prob["coords"].shape[0] * prob["dim"]
        Fs = []
        for f in forces:
            F = np.zeros(n)
            s.assemble_load(f, F)
            Fs.append(F)
        s.close()
        loads.append(Fs)
    n_solves = sum(len(F) for F in loads)
    dofs = [prob["coords"].shape[0] * prob["dim"] for prob, _ in reqs]

    def run(slots, precision, rate=None, batch=False):
        srv = vasmg.Server(slots=slots, precision=precision, batch=batch)
        rs = meshgen.Stream(77)
        gaps = -np.log(1.0 - rs.uniform(len(reqs))) / rate if rate else np.zeros(len(reqs))
        t0 = time.perf_counter()
        tickets, outs = [], []
        t_next = t0
        for (prob, _), Fs, g in zip(reqs, loads, gaps):
            t_next += g
            while time.perf_counter() < t_next:
                time.sleep(min(0.001, max(0.0, t_next - time.perf_counter())))
            Us = [np.zeros_like(F) for F in Fs]
            outs.append(Us)
            tickets.append(srv.submit(prob, Fs, Us))
        stats = [srv.poll(t, -1) for t in tickets]
        t1 = time.perf_counter()
        srv.close()
        lat = np.array([st["latency_ms"] for st in stats])
        ok = all(st["status"] == 0 for st in stats)
        return {"solves_per_s": n_solves / (t1 - t0), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "all_converged": ok,
                "iterations": int(sum(st["iterations"] for st in stats))}

    run(4, "fp32")  # warm-up: kernels loaded, graphs paths exercised
    single = run(1, "fp32")
    cap_rps = len(reqs) / (n_solves / single["solves_per_s"])
    closed = run(4, "fp32")
    fp64_single = run(1, "fp64")
    loads_out = {}
    for frac in (0.5, 0.8, 0.95):
        loads_out[str(frac)] = run(4, "fp32", rate=frac * cap_rps)
    # the batched executor: every ready request's next right-hand side in one
    # round of vasmg_solve_batch (one launch per level and phase for all)
    batched = {"closed_loop": run(4, "fp32", batch=True), "offered_load": {}}
    for frac in (0.5, 0.8, 0.95):
        batched["offered_load"][str(frac)] = run(4, "fp32", rate=frac * cap_rps, batch=True)
    return {"requests": len(reqs), "solves": n_solves, "dofs_min": int(min(dofs)), "dofs_max": int(max(dofs)),
            "slots": 4, "precision": "fp32 V-cycle, fp64 CG",
            "single_stream": single, "closed_loop": closed, "fp64_single_stream": fp64_single,
            "offered_load": loads_out, "batched": batched, "capacity_requests_per_s": cap_rps,
            "recipe": "Poisson arrivals (seed 5/77), mixed 2D/3D jittered P1, 5k-500k dofs log-uniform, "
                      "E~U[1,100], nu~U[0.2,0.45], 1-8 body-force loads each, tol 1e-6"}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = SAMPLE_N.get(args.workload, 32)
    vals, nfree, _ = cpu_oracle_run(args.workload, n, args.warmup + args.steps)
    timed = vals[args.warmup:] if len(vals) > args.warmup else vals
    total_work = sum(v[0] * v[2] for v in timed)
    total_t = sum(v[2] for v in timed)
    value = total_work / total_t
    side = f"{n}^3" if args.workload.startswith("cube") else f"{n}x{n}"
    sample = (f"{args.workload} recipe at {side} vertices ({nfree} free dofs), one full solve to {TOL} per step, "
              f"1 thread, CPU {cpu_model()}")
    line = {"impl": "reference", "metric": "V-ASMG-PCG MDOF*iter/s to 1e-6 rel. residual", "value": value,
            "unit": "MDOF*iter/s", "n_gpus": args.gpus, "steps": len(timed), "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / len(timed), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload} (CPU oracle sample {side})", "iterations": timed[0][1]},
            "cpu_baseline": {"value": value, "unit": "MDOF*iter/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": value, "unit": "MDOF*iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fp64_roof(vasmg):
    """Measured FP64 FMA rate (TFLOP/s) of this GPU, the arithmetic roof of the
    FP64 kernels."""
    tf, ms = vasmg.vasmg_probe_fp64_rate()
    return {"tflops": tf, "kernel_ms": ms, "how": "independent FMA chains on every SM, CUDA events, mean of 5 launches"}


def spmv64_flops(s, vasmg):
    """Algorithmic FP64 flops of one level-0 SpMV with the p.q product: 2 d^2
    per stored block (diagonal included) + 2 per dof."""
    d = 2 if s.dim == 2 else 3
    nv, nnzb, _ = vasmg.vasmg_level_info(s.h, 0)
    return 2.0 * d * d * nnzb + 2.0 * nv * d


def multi_rhs_run(s, F, n, nfree, k, dev, peaks):
    """k right-hand sides on the headline hierarchy: the first is the
    workload's load, the others body-force loads in seeded random directions.
    Times one vasmg_solve_multi call against the k single solves (CUDA
    events), checks that every solution is bitwise the single one, and times
    the region kernels with k right-hand sides per launch."""
    import torch

    from paper_2505_09064_gb300 import meshgen, vasmg

    rs = meshgen.Stream(123)
    d = s.dim
    Fs = [F]
    for i in range(1, k):
        Fi = torch.zeros(n, dtype=torch.float64, device=dev)
        s.assemble_load(rs.uniform(d, -1.0, 1.0), Fi)
        Fs.append(Fi)
    Us = [torch.zeros_like(Fi) for Fi in Fs]
    s.solve_multi(Fs, Us, TOL)  # warm-up: buffers and graph of the pass
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    rc, sts, _ = s.solve_multi(Fs, Us, TOL)
    ev1.record()
    torch.cuda.synchronize()
    ms_multi = ev0.elapsed_time(ev1)
    launches_multi = vasmg.vasmg_last_launch_count(s.h)
    its = [st.iterations for st in sts]
    U1s = [torch.zeros_like(F) for _ in range(k)]
    single_its = []
    torch.cuda.synchronize()
    ev0.record()
    for i in range(k):
        rc1, st1, _ = s.solve(Fs[i], U1s[i], TOL)
        single_its.append(st1.iterations)
    ev1.record()
    torch.cuda.synchronize()
    ms_single = ev0.elapsed_time(ev1)
    bitwise = all(bool(torch.equal(U1s[i], Us[i])) for i in range(k))
    del U1s
    work = float(nfree * sum(its))
    out = {"k": k, "value": work / (ms_multi / 1e3) / 1e6, "unit": "MDOF*iter/s", "ms": ms_multi,
           "solves_per_s": k / (ms_multi / 1e3), "iterations": its, "gpu_launches": launches_multi,
           "single_solves": {"value": work / (ms_single / 1e3) / 1e6, "ms": ms_single, "iterations": single_its},
           "speedup_vs_single": ms_single / ms_multi, "bitwise_equal_to_single": bitwise and its == single_its}
    # the region kernels with k right-hand sides per launch: operator bytes
    # once, vector bytes k times
    kern = {}
    nlev = vasmg.vasmg_num_levels(s.h)
    for l in range(nlev - 1):
        if vasmg.vasmg_level_info(s.h, l)[0] <= TAIL_NV:
            break
        for name, which in (("fwd_sweep", vasmg.KERNEL_FWD_SWEEP), ("residual", vasmg.KERNEL_RESIDUAL),
                            ("bwd_sweep", vasmg.KERNEL_SWEEP)):
            kms, kb = vasmg.vasmg_time_kernel_multi(s.h, which, l, k, 5)
            kern[f"{name}_l{l}"] = {"ms": kms, "bytes": kb, "gbs": kb / (kms / 1e3) / 1e9,
                                    "frac": kb / (kms / 1e3) / 1e9 / peaks["hbm_gbs"]}
    out["launches"] = kern
    top = max(kern, key=lambda q: kern[q]["ms"])
    out["roofline"] = {"kernel": top, "achieved": kern[top]["gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": kern[top]["frac"], "bytes_per_launch": kern[top]["bytes"], "k": k}
    return out


def ours(args):
    import torch

    from paper_2505_09064_gb300 import meshgen, vasmg

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream().cuda_stream
    if args.fp64_peak:
        if rank == 0:
            print(json.dumps({"fp64_fma": fp64_roof(vasmg)}), flush=True)
        return

    def make(workload, precision, threshold=0):
        prob = sample_problem(workload, args.side) if args.side else meshgen.make_problem(workload)
        n = prob["coords"].shape[0] * prob["dim"]
        nfree = n - prob["dirichlet_dofs"].size
        s = vasmg.Solver(prob, precision=precision, stream=stream, use_graph=not args.no_graph,
                         threshold=threshold, autotune=not args.no_autotune)
        F = torch.zeros(n, dtype=torch.float64, device=dev)
        s.assemble_load(prob["body_force"], F)
        U = torch.zeros_like(F)
        for _ in range(args.warmup):
            s.solve(F, U, TOL)
        torch.cuda.synchronize()
        return s, F, U, n, nfree

    def timed(s, F, U, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters, launches = [], 0
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(steps):
            rc, st, _ = s.solve(F, U, TOL)
            assert rc == 0, rc
            iters.append(st.iterations)
            launches += vasmg.vasmg_last_launch_count(s.h)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        if world > 1:
            torch.distributed.barrier()
        return ms, iters, launches, st

    def line_of(workload, precision, steps, threshold=0, keep=False):
        """A secondary line: value, iterations and ms per solve of one
        configuration (timed alone, CUDA events)."""
        s2, F2, U2, n2, nf2 = make(workload, precision, threshold)
        ms2, it2, _, st2 = timed(s2, F2, U2, steps)
        nb = [vasmg.vasmg_level_info(s2.h, l)[1] for l in range(vasmg.vasmg_num_levels(s2.h))]
        out = {"value": nf2 * sum(it2) / (ms2 / 1e3) / 1e6, "unit": "MDOF*iter/s", "precision": precision,
               "iterations": it2[0], "ms_per_solve": ms2 / len(it2), "solves": len(it2), "dofs": n2,
               "free_dofs": nf2, "setup_ms": st2.setup_ms, "levels": len(nb), "op_complexity": sum(nb) / nb[0]}
        if threshold:
            out["leaf_threshold"] = threshold
        if keep:
            return out, (s2, U2)
        s2.close()
        return out, None

    if args.profile_kernel:
        kind, level = args.profile_kernel.split(":")
        which = {"spmv64": vasmg.KERNEL_SPMV64, "sweep": vasmg.KERNEL_SWEEP, "fwd_sweep": vasmg.KERNEL_FWD_SWEEP,
                 "residual": vasmg.KERNEL_RESIDUAL, "restrict": vasmg.KERNEL_RESTRICT,
                 "prolong": vasmg.KERNEL_PROLONG, "tail": vasmg.KERNEL_TAIL}[kind]
        s, F, U, n, nfree = make(args.workload, args.precision)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        if args.profile_k > 1:
            kms, kbytes = vasmg.vasmg_time_kernel_multi(s.h, which, int(level), args.profile_k, 1)
        else:
            kms, kbytes = vasmg.vasmg_time_kernel(s.h, which, int(level), 1)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        if rank == 0:
            print(json.dumps({"profile_kernel": args.profile_kernel, "k": args.profile_k, "workload": args.workload,
                              "side": args.side, "precision": args.precision, "ms": kms, "algorithmic_bytes": kbytes,
                              "lanes_per_row": [int(g) for g in s.export(vasmg.EXPORT_LANES, 0, np.int32)],
                              "level_vertices": [vasmg.vasmg_level_info(s.h, l)[0]
                                                 for l in range(vasmg.vasmg_num_levels(s.h))]}), flush=True)
        s.close()
        return
    # headline
    s, F, U, n, nfree = make(args.workload, args.precision)
    clocks = ClockSampler(local)
    clocks.start()
    if args.solve_only:
        torch.cuda.profiler.start()  # the solves alone, for ncu --profile-from-start off
    ms, iters, launches, st = timed(s, F, U, args.steps)
    if args.solve_only:
        torch.cuda.profiler.stop()
    clk = clocks.stop()
    ms, work = reduce_over_ranks(ms, float(nfree * sum(iters)), dev)
    value = work / (ms / 1e3) / 1e6
    if args.solve_only:
        if rank == 0:
            print(json.dumps({"metric": "V-ASMG-PCG MDOF*iter/s to 1e-6 rel. residual", "value": value,
                              "unit": "MDOF*iter/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                              "ms_per_step": ms / args.steps, "iterations": iters[0], "gpu_launches": launches,
                              "graph": not args.no_graph, "solve_only": True, "workload": args.workload,
                              "side": args.side,
                              "precision": args.precision, "clocks": clk,
                              "lanes_per_row": [int(g) for g in s.export(vasmg.EXPORT_LANES, 0, np.int32)]}),
                  flush=True)
        s.close()
        return
    # roofline: every kernel of one PCG iteration timed alone on the library's
    # stream (CUDA events, mean over repetitions); the one with the largest
    # time per iteration is the dominant kernel
    peaks, peak_src = load_peaks()
    nlev = vasmg.vasmg_num_levels(s.h)
    kernels = {"spmv64_sell": vasmg.vasmg_time_kernel(s.h, vasmg.KERNEL_SPMV64, 0, 20)}
    lt = nlev - 1
    for l in range(nlev - 1):
        if levels_vertices(s, l) <= TAIL_NV:
            lt = l
            break
        kernels[f"fwd_sweep_l{l}"] = vasmg.vasmg_time_kernel(s.h, vasmg.KERNEL_FWD_SWEEP, l, 10)
        kernels[f"residual_l{l}"] = vasmg.vasmg_time_kernel(s.h, vasmg.KERNEL_RESIDUAL, l, 10)
        kernels[f"restrict_l{l}"] = vasmg.vasmg_time_kernel(s.h, vasmg.KERNEL_RESTRICT, l, 10)
        kernels[f"prolong_l{l}"] = vasmg.vasmg_time_kernel(s.h, vasmg.KERNEL_PROLONG, l, 10)
        kernels[f"bwd_sweep_l{l}"] = vasmg.vasmg_time_kernel(s.h, vasmg.KERNEL_SWEEP, l, 10)
    if lt < nlev - 1:
        kernels[f"tail_l{lt}"] = vasmg.vasmg_time_kernel(s.h, vasmg.KERNEL_TAIL, lt, 10)
    vc_ms, vc_bytes = vasmg.vasmg_time_kernel(s.h, vasmg.KERNEL_VCYCLE, 0, 10)
    top = max(kernels, key=lambda k: kernels[k][0])
    k_ms, k_bytes = kernels[top]
    achieved = k_bytes / (k_ms / 1e3) / 1e9
    f64 = fp64_roof(vasmg)
    sp_ms, sp_bytes = kernels["spmv64_sell"]
    sp_flops = spmv64_flops(s, vasmg)
    spmv_roofs = {"ms": sp_ms, "bytes": sp_bytes, "gbs": sp_bytes / (sp_ms / 1e3) / 1e9,
                  "hbm_frac": sp_bytes / (sp_ms / 1e3) / 1e9 / peaks["hbm_gbs"], "flops": sp_flops,
                  "tflops": sp_flops / (sp_ms / 1e3) / 1e12,
                  "fp64_frac": sp_flops / (sp_ms / 1e3) / 1e12 / f64["tflops"]}
    # e2e: pinned host F and U, copies inside the timed region
    Fh = F.cpu().pin_memory()
    Uh = torch.zeros_like(Fh).pin_memory()
    for _ in range(2):
        s.solve(Fh.numpy(), Uh.numpy(), TOL)
    t0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(args.steps):
        rc, st2, _ = s.solve(Fh.numpy(), Uh.numpy(), TOL)
        e2e_iters += st2.iterations
    e2e_s = time.perf_counter() - t0
    e2e_ms, e2e_work = reduce_over_ranks(e2e_s * 1e3, float(nfree * e2e_iters), dev)
    e2e = e2e_work / (e2e_ms / 1e3) / 1e6
    # several right-hand sides per launch (vasmg_solve_multi): 8 loads of
    # the same mesh solved together against the same 8 solved one by one
    multi = None
    if args.precision != "fp64" and world == 1:
        multi = multi_rhs_run(s, F, n, nfree, 8, dev, peaks)
    levels = [vasmg.vasmg_level_info(s.h, l) for l in range(vasmg.vasmg_num_levels(s.h))]
    lanes = [int(g) for g in s.export(vasmg.EXPORT_LANES, 0, np.int32)]
    dense = [int(v) for v in s.export(vasmg.EXPORT_DENSE, 0, np.int64)]
    # slots of the staged backward-sweep copy per block, per region level (0: unstaged)
    staged_pad = []
    for l in range(len(lanes)):
        if lanes[l] == 0:
            break
        sx = s.export(vasmg.EXPORT_STAGED, l, np.int64)
        staged_pad.append(round(float(sx[2]) / float(sx[3]), 3) if sx[3] > 0 else 0.0)
    setup_ms = st.setup_ms
    op_cx = st.op_complexity
    # the plain FP64 path on the same workload, with the headline solution's
    # distance from it (the FP64 path matches the FP64 oracle to 1e-10 on the
    # parity cases)
    fp64 = None
    extra = max(1, min(args.steps, 3))
    if args.precision != "fp64":
        fp64, keep = line_of(args.workload, "fp64", extra, keep=True)
        s64, U64 = keep
        fp64["rel_error_of_headline_solution"] = float((U - U64).abs().max().item() /
                                                       max(U64.abs().max().item(), 1e-300))
        fp64["spmv64"] = {"ms": vasmg.vasmg_time_kernel(s64.h, vasmg.KERNEL_SPMV64, 0, 20)[0]}
        s64.close()
    # the other configurations, each on its own
    others = None
    if not args.no_others and world == 1:
        s.close()
        s = None
        others = {}
        for wl in ("square64", "square1024_checker", "cube64"):
            if wl == args.workload:
                continue
            pr = DEFAULT_PRECISION[wl]
            entry = {pr: line_of(wl, pr, extra)[0]}
            if pr != "fp64":
                entry["fp64"] = line_of(wl, "fp64", extra)[0]
            if wl == "square1024_checker":
                # leaf threshold 8 instead of the paper's 4: fewer, sparser coarse levels
                entry["leaf_threshold_8"] = line_of(wl, pr, extra, threshold=8)[0]
            others[wl] = entry
    serving = None
    if not args.no_serving:
        serving = serving_run(stream)
    line = {"metric": "V-ASMG-PCG MDOF*iter/s to 1e-6 rel. residual", "value": value, "unit": "MDOF*iter/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f64 CG + f32 V-cycle", "bf16": "f64 CG + f32/bf16 V-cycle"}[
                args.precision],
            "data": "synthetic",
            "config": {"workload": args.workload, "dofs": n, "free_dofs": nfree, "iterations": iters[0],
                       "ms_per_solve": ms / args.steps, "precision": args.precision, "tol": TOL,
                       "levels": len(levels), "level_vertices": [lv[0] for lv in levels],
                       "level_blocks": [lv[1] for lv in levels], "level_colours": [lv[2] for lv in levels],
                       "op_complexity": op_cx, "lanes_per_row": lanes, "dense_level": dense,
                       "staged_slots_per_block": staged_pad,
                       "setup_ms": setup_ms, "l2": "operators > L2 (no flush needed)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "limiter": "latency" if top.startswith("tail") else "latency/HBM",
                         "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": TRAFFIC.get((args.workload, top)),
                         "kernel": top, "peak_source": peak_src, "launch_ms": k_ms, "algorithmic_bytes": k_bytes,
                         "launches": {k: {"ms": v[0], "bytes": v[1], "gbs": v[1] / (v[0] / 1e3) / 1e9}
                                      for k, v in kernels.items()},
                         "vcycle": {"ms": vc_ms, "bytes": vc_bytes, "gbs": vc_bytes / (vc_ms / 1e3) / 1e9},
                         "fp64_fma": f64, "spmv64": spmv_roofs},
            "e2e": {"value": e2e, "unit": "MDOF*iter/s", "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
            "gpu_launches": launches, "clocks": clk, "fp64_path": fp64, "multi_rhs": multi,
            "other_workloads": others, "serving": serving}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ns = SAMPLE_N.get(args.workload, 32)
        side = f"{ns}^3" if args.workload.startswith("cube") else f"{ns}x{ns}"
        model = cpu_model()
        vals, nf, _ = cpu_oracle_run(args.workload, ns, 1)
        v = vals[-1]
        line["cpu_baseline"] = {"value": v[0], "unit": "MDOF*iter/s", "cores": 1, "kind": "oracle",
                                "cpu_model": model, "nproc": os.cpu_count(),
                                "sample": f"{args.workload} recipe at {side} vertices ({nf} free dofs), "
                                          f"one full solve to {TOL}, {v[1]} iterations, {v[2]:.1f} s, 1 thread"}
        # second CPU line: the same oracle source built with OpenMP, its
        # independent row loops on every host core (bitwise the same solve)
        vals, nf, th = cpu_oracle_run(args.workload, ns, 2, threads=os.cpu_count() or 1)
        v = max(vals)
        line["cpu_baseline_parallel"] = {
            "value": v[0], "unit": "MDOF*iter/s", "cores": th, "kind": "oracle, OpenMP build", "cpu_model": model,
            "sample": f"as cpu_baseline, {v[1]} iterations, {th} threads (colour, y = A x and prolongation row "
                      f"loops parallel; reductions serial), best of 2 solves"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if s is not None:
        s.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
