"""Benchmark: FD-preconditioned MINRES on the isogeometric Stokes system.

One step = P_D-preconditioned MINRES (tol 1e-8, x0 = 0) on a batch of
right-hand sides of the named workload, through the library's C ABI
(every stage of the hot path: Kronecker matvec, FD preconditioner apply,
MINRES recurrences and inner products). Default workload: 3D unit cube,
Taylor-Hood, p=3, 64^3 elements (6,740,830 DoF), 16 seeded N(0,1)
right-hand sides. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FD applies/s (GDoF/s) and MINRES solves/s vs plain FP64 at stated error; p99 latency"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 1.25     # GB300 FP64 (DFMA) nominal, profiling recipe table
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 flops x max SM clock
TF32_OVER_BF16 = 1.1 / 2.25    # nominal dense TF32 / BF16 ratio


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="cube_th_p3_64")
    ap.add_argument("--fd", default="auto", choices=["auto", "f64", "tf32"])
    ap.add_argument("--matvec", default="df64", choices=["f64", "df64"],
                    help="matvec arithmetic inside the iterations (true residual always FP64)")
    ap.add_argument("--nrhs", type=int, default=0, help="right-hand sides per step (default: the workload's)")
    ap.add_argument("--maxit", type=int, default=400)
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def workload(name):
    import synth
    w = dict(synth.WORKLOADS[name])
    return w


def describe(name, w, nrhs):
    n = "x".join(str(v) for v in w["n_el"])
    return (f"{name}: {w['dim']}D unit {'cube' if w['dim'] == 3 else 'square'}, {w['disc']} IGA, pressure degree "
            f"p={w['p']}, {n} elements, {nrhs} seeded N(0,1) right-hand sides (pressure part mean-free), "
            f"P_D-MINRES tol 1e-8 from x0=0")


def peaks():
    try:
        return json.load(open(MEASURED_PEAKS))
    except (OSError, ValueError):
        return {}


def cpu_oracle_sample(w, seeds, iters_per_solve, k_iters=2):
    """The oracle as it stands on the host cores: k_iters MINRES iterations at
    full workload size on one right-hand side, scaled to solves/s with the
    iteration count of a full solve."""
    import numpy as np

    import synth
    from oracle import minres, stokes
    knots = [synth.open_uniform_knots(n, w["p"]) for n in w["n_el"]]
    S = stokes.build(knots, w["p"], w["disc"])
    b = synth.rhs(seeds[0], S.block_sizes)
    t0 = time.perf_counter()
    minres.minres(lambda v: stokes.matvec(S, v), b, lambda v: stokes.apply_PD_inv(S, v), tol=0.0, maxit=k_iters)
    dt = time.perf_counter() - t0
    t_iter = dt / (k_iters + 1)          # k iterations + the initial matvec/apply
    value = 1.0 / (t_iter * iters_per_solve)
    return dict(value=value, unit="solves/s", cores=os.cpu_count(), kind="oracle",
                sample=(f"{k_iters} MINRES iterations of the NumPy/SciPy FP64 oracle on 1 right-hand side at "
                        f"full size ({dt:.1f} s incl. the initial matvec+apply), per-iteration time x "
                        f"{iters_per_solve:.1f} iterations per solve; BLAS threads = default (all cores)"),
                seconds=dt, t_iter_s=t_iter)


# ------------------------------------------------------------------ reference arm (oracle on CPU)

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.workload)
    nrhs = args.nrhs or len(w["seeds"])
    iters = 56.0   # iterations per solve used for scaling (cube TH P_D-MINRES, paper Table cube_TH)
    for _ in range(args.warmup):
        cpu_oracle_sample(w, w["seeds"], iters, k_iters=1)
    vals, secs = [], []
    for _ in range(args.steps):
        r = cpu_oracle_sample(w, w["seeds"], iters, k_iters=1)
        vals.append(r["value"])
        secs.append(r["t_iter_s"] * iters)
    value = statistics.median(vals)
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": describe(args.workload, w, 1), "nrhs": 1},
           "cpu_baseline": {"value": value, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": "per step: 1 MINRES iteration (plus the initial matvec and apply) of the "
                                      "FP64 oracle at full size on 1 RHS, scaled by 56 iterations per solve"},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ GPU arm

def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1712_00403_gb300 as fd
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = workload(args.workload)
    nrhs = args.nrhs or len(w["seeds"])
    if args.fd == "auto":
        prec = fd.FD_TF32X3 if getattr(fd, "HAS_TC", False) else fd.FD_F64
    else:
        prec = fd.FD_F64 if args.fd == "f64" else fd.FD_TF32X3
    knots = synth.knots_for(w)
    t_setup = time.perf_counter()
    mv = fd.MV_DF64 if args.matvec == "df64" else fd.MV_F64
    P = fd.Stokes(knots, w["p"], disc=fd.TH if w["disc"] == "TH" else fd.RT, fd_precision=prec, max_rhs=nrhs,
                  matvec_precision=mv)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    # weak scaling: every rank solves its own batch (seeds shifted by rank)
    seeds = [w["seeds"][j % len(w["seeds"])] + 1000 * rank for j in range(nrhs)]
    B = np.stack([synth.rhs(s, P.block_sizes) for s in seeds])
    b = torch.tensor(B.reshape(-1), device=dev)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()

    def step():
        x.zero_()
        return P.solve(b, x, tol=1e-8, maxit=args.maxit, stream=stream)

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    P.set_timing(True)
    launches0 = fd.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
    launches = fd.kernel_launches() - launches0
    tm = P.get_timing()
    P.set_timing(False)
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    clocks = clk.summary()
    total_solves = args.steps * nrhs * world
    value = total_solves / (ms / 1e3)

    iters = [i["iterations"] for inf in infos for i in inf]
    statuses = sorted(set(i["status"] for inf in infos for i in inf))
    true_res = max(i["true_rel_res"] for inf in infos for i in inf)

    # FD apply throughput (untimed part of the step, reported beside it)
    s = torch.empty_like(b)
    for _ in range(2):
        P.apply_prec(b, s, stream=stream)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    a0.record(stream)
    for _ in range(reps):
        P.apply_prec(b, s, stream=stream)
    a1.record(stream)
    torch.cuda.synchronize()
    ms_apply = a0.elapsed_time(a1) / reps
    applies_per_s = nrhs / (ms_apply / 1e3)
    apply_err = None
    if prec != fd.FD_F64:
        P64 = fd.Stokes(knots, w["p"], disc=fd.TH if w["disc"] == "TH" else fd.RT, fd_precision=fd.FD_F64,
                        max_rhs=1)
        s64 = torch.empty(P.n_total, dtype=torch.float64, device=dev)
        P64.apply_prec(b[:P.n_total].contiguous(), s64, stream=stream)
        torch.cuda.synchronize()
        apply_err = float(torch.linalg.norm(s[:P.n_total] - s64) / torch.linalg.norm(s64))
        P64.close()

    # roofline of the dominant phase (timed live inside the timed region)
    pk = peaks()
    per_mv = tm["ms_matvec"] / max(tm["n_matvec"], 1)
    per_pc = tm["ms_prec"] / max(tm["n_prec"], 1)
    if per_mv >= per_pc and mv == fd.MV_F64:
        kern, flops, t_ms = "stokes_matvec_f64 (banded Kronecker mode products)", P.flops_matvec * nrhs, per_mv
        peak = FP64_NOMINAL_TFLOPS
        peak_note = "FP64 DFMA nominal 1.25 TFLOP/s (recipe table; measured DFMA chain 1.20)"
        bound = "alu"
    elif per_mv >= per_pc:
        # double-float: 12 FP32 operations per banded multiply-add (exact product + TwoSum)
        kern = "stokes_matvec_df64 (banded Kronecker mode products, FP32-pair arithmetic)"
        flops, t_ms = P.flops_matvec * nrhs * 6.0, per_mv
        peak = FP32_NOMINAL_TFLOPS
        peak_note = ("FP32 ALU: 152 SMs x 128 FP32 lanes x 2070 MHz = 80.5 TFLOP/s nominal (FFMA chain measured 75); "
                     "achieved counts 12 FP32 ops per multiply-add of the plan")
        bound = "alu"
    else:
        kern, flops, t_ms = "fd_apply", P.flops_apply * nrhs, per_pc
        if prec == fd.FD_F64:
            peak, bound = FP64_NOMINAL_TFLOPS, "alu"
            peak_note = "FP64 DFMA nominal 1.25 TFLOP/s (recipe table; measured DFMA chain 1.20)"
        else:
            peak = pk.get("bf16_tflops_sustained", 1748.4) * TF32_OVER_BF16
            bound = "tensor"
            peak_note = "TF32 = measured bf16 sustained x nominal TF32/BF16 ratio"
            flops *= 3  # three split products per contraction
    achieved = flops / (t_ms / 1e3) / 1e12
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": kern, "ms_per_launch": t_ms, "peak_source": peak_note}

    # end to end through the host-pointer entry point (pinned host buffers)
    bh = torch.empty(b.numel(), dtype=torch.float64, pin_memory=True)
    bh.copy_(b.cpu())
    xh = torch.zeros(b.numel(), dtype=torch.float64, pin_memory=True)
    bn, xn = bh.numpy(), xh.numpy()
    e2e_steps = max(1, args.steps // 3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        xn[:] = 0.0
        P.solve_host(bn, xn, tol=1e-8, maxit=args.maxit, stream=stream)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": e2e_steps * nrhs * world / e2e_s, "unit": "solves/s",
           "h2d_bytes_per_step": 2 * b.numel() * 8, "d2h_bytes_per_step": b.numel() * 8}

    cpu = None
    if rank == 0 and world == 1:
        cpu = cpu_oracle_sample(w, w["seeds"], float(np.mean(iters)), k_iters=2)
        cpu.pop("seconds", None)
        cpu.pop("t_iter_s", None)

    if rank == 0:
        dtype = "f64" if prec == fd.FD_F64 else "f64+tf32x3"
        if mv == fd.MV_DF64:
            dtype += " (matvec df64)"
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": dtype, "data": "synthetic",
               "config": {"workload": describe(args.workload, w, nrhs), "nrhs_per_gpu": nrhs,
                          "fd_precision": "f64" if prec == fd.FD_F64 else "tf32x3",
                          "matvec": ("double-float (FP32 pairs, 48-bit significand) in the iterations; "
                                     "true residual in FP64") if mv == fd.MV_DF64 else "FP64",
                          "n_total": P.n_total,
                          "l2": "inputs larger than L2 (each step streams %d x %.0f MB vectors)" % (
                              nrhs, P.n_total * 8 / 1e6),
                          "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
               "minres": {"iterations_min": min(iters), "iterations_max": max(iters), "status": statuses,
                          "true_rel_res_max": true_res},
               "fd_apply": {"applies_per_s": applies_per_s, "gdof_per_s": applies_per_s * P.n_total / 1e9,
                            "ms_per_batch": ms_apply, "rel_err_vs_f64": apply_err},
               "phases_ms_per_iter": {"matvec": per_mv, "prec": per_pc,
                                      "vector": tm["ms_vector"] / max(tm["n_matvec"], 1)},
               "setup_s": t_setup, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(out), flush=True)
    P.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
