"""Benchmark: FD-preconditioned MINRES on the isogeometric Stokes system.

One step = P_D-preconditioned MINRES (tol 1e-8, x0 = 0) on a batch of
right-hand sides of the named workload, through the library's C ABI
(every stage of the hot path: Kronecker matvec, FD preconditioner apply,
MINRES recurrences and inner products). Default workload: 3D unit cube,
Taylor-Hood, p=3, 64^3 elements (6,740,830 DoF), 16 seeded N(0,1)
right-hand sides. Prints one JSON line (rank 0).

Other workloads (--workload): mapped_th_p3_32 (sine-bump map, variable
viscosity, P_D^G, FP64 CSR operator, 4 right-hand sides), annulus_th_p3_32
(the eighth of a thick annulus, nu = 1, otherwise the same; --matrix-free
selects the sum-factorized operator on either), batched_64 (64
uneven unit-cube instances in grouped launches; split-TF32 and FP64 FD
compared) and serving (Poisson arrivals swept over rates through the request
server; p50/p99 latency).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--workload NAME]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FD applies/s (GDoF/s) and MINRES solves/s vs plain FP64 at stated error; p99 latency"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 1.25     # GB300 FP64 (DFMA) nominal, profiling recipe table
FP32_LANE_TOPS = 152 * 128 * 2.070e9 / 1e12   # SMs x FP32 lanes x max SM clock: lane operations per second
TF32_OVER_BF16 = 1.1 / 2.25    # nominal dense TF32 / BF16 ratio
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant matvec kernel from
# ncu captures of the kernels as they stand: k_band_df summed over the 24 launches of one
# double-float matvec of the 40^3 cube (16 RHS, 1,673,830 entries each), scaled to a workload
# by its entry count (every launch streams operands proportional to it); k_spmv_df per launch
# of the 32^3 mapped operator at 4 RHS, the bench's own size.
MATVEC_TRAFFIC = {"k_band_df": {"bytes": 5.6576e9, "entries": 1_673_830, "nrhs": 16, "launches": 24},
                  # captured on the 16^3 mapped cube (168,894,405 nonzeros), scaled by nonzero count
                  "k_spmv_df": {"bytes": 2.0534e9, "nnz": 168_894_405, "nrhs": 4, "launches": 1}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="cube_th_p3_64")
    ap.add_argument("--fd", default="auto", choices=["auto", "f64", "tf32", "bf16"])
    ap.add_argument("--matvec", default="df64", choices=["f64", "df64"],
                    help="matvec arithmetic inside the iterations (true residual always FP64)")
    ap.add_argument("--nrhs", type=int, default=0, help="right-hand sides per step (default: the workload's)")
    ap.add_argument("--maxit", type=int, default=400)
    ap.add_argument("--solver", default="minres", choices=["minres", "gmres-pt", "gmres-pc"],
                    help="P_D-MINRES (the default), or GMRES with the block triangular P_T / constraint P_C")
    ap.add_argument("--restart", type=int, default=60, help="GMRES Krylov basis size")
    ap.add_argument("--matrix-free", action="store_true",
                    help="mapped workloads: sum-factorized matvec in the iterations instead of the CSR SpMV")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the plain-FP64 leg (FD apply and matvec in FP64; batched: the FP64-FD batch)")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the plain-FP64 leg")
    ap.add_argument("--serving-max-active", type=int, default=16,
                    help="most requests the server advances together (serving workload)")
    ap.add_argument("--serving-iters", type=int, default=4,
                    help="MINRES iterations per scheduler step (serving workload)")
    ap.add_argument("--serving-nel3-max", type=int, default=96,
                    help="largest elements per direction of the served 3D instances (default: the batched range 16..96)")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle timing (profiling runs of the GPU path)")
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
        sm, mx, pw, reasons = [], [], [], set()
        for line in self.f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            try:
                pw.append(float(parts[3]))
            except ValueError:
                pass
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "sm_min_mhz": min(sm),
                "power_w_median": statistics.median(pw) if pw else None}


# ------------------------------------------------------------------ helpers

# ------------------------------------------------------------------ replicas (one process per GPU)

class Replicas:
    """Multi-GPU layout: the path does not shard, so N GPUs run N independent replicas,
    one process per GPU under torchrun (WORLD_SIZE / RANK / LOCAL_RANK from the
    environment). Each rank solves its own right-hand sides (seeds shifted by
    SEED_STRIDE x rank) and nothing crosses ranks on the data path. The collectives are
    the timing ones only: a barrier on both sides of a timed region, the max over ranks
    of its duration and the sum over ranks of the units solved, so that the job's value
    is all units / the slowest rank's time. backend "nccl" reduces on the rank's GPU;
    "gloo" on the host (the multi-process tests run it on CPU)."""

    SEED_STRIDE = 1000

    def __init__(self, backend="nccl", env=None, timeout_s=None):
        env = os.environ if env is None else env
        self.world = int(env.get("WORLD_SIZE", "1"))
        self.rank = int(env.get("RANK", "0"))
        self.local = int(env.get("LOCAL_RANK", "0"))
        self.backend = backend
        if backend == "nccl":
            import torch
            torch.cuda.set_device(self.local)
        if self.world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                if timeout_s is None:
                    dist.init_process_group(backend)
                else:
                    import datetime
                    # a collective that a departed rank never joins fails after this long
                    dist.init_process_group(backend, timeout=datetime.timedelta(seconds=timeout_s))
            if dist.get_world_size() != self.world or dist.get_rank() != self.rank:
                raise RuntimeError("process group (%d of %d) disagrees with RANK/WORLD_SIZE (%d of %d)" % (
                    dist.get_rank(), dist.get_world_size(), self.rank, self.world))

    @property
    def parallelism(self):
        return f"replicas x{self.world}" if self.world > 1 else "1 GPU"

    def seed(self, s):
        """This rank's copy of a workload seed."""
        return s + self.SEED_STRIDE * self.rank

    def seeds(self, base, n):
        """n right-hand-side seeds of this rank: the workload's list cycled, then shifted."""
        return [self.seed(base[j % len(base)]) for j in range(n)]

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def reduce(self, values, op):
        """Floats reduced elementwise over ranks; op "max" or "sum" (FP64 on the wire)."""
        vals = [float(v) for v in values]
        if self.world == 1:
            return vals
        import torch
        import torch.distributed as dist
        dev = torch.device("cuda", torch.cuda.current_device()) if self.backend == "nccl" else torch.device("cpu")
        t = torch.tensor(vals, dtype=torch.float64, device=dev)
        dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[op])
        return [float(v) for v in t.cpu()]

    def max(self, v):
        return self.reduce([v], "max")[0]

    def sum(self, v):
        return self.reduce([v], "sum")[0]

    def job_rate(self, units, seconds):
        """Whole-job throughput: this rank's units summed over ranks / the slowest rank's seconds."""
        tot, = self.reduce([units], "sum")
        worst, = self.reduce([seconds], "max")
        return tot / worst

    def close(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()


def workload(name):
    import synth
    w = dict(synth.WORKLOADS[name])
    return w


def describe(name, w, nrhs, matrix_free=False):
    n = "x".join(str(v) for v in w["n_el"])
    if w.get("geometry") in ("sine_bump", "annulus"):
        op = "matrix-free operator (sum factorization, no CSR)" if matrix_free else "FP64 CSR operator"
        dom = ("3D cube mapped by x = xi + 0.1 sin(pi xi1) sin(pi xi2) sin(pi xi3) (1,1,1), viscosity "
               "1 + 0.5 sin(2 pi x1) cos(2 pi x2)" if w["geometry"] == "sine_bump" else
               "eighth of a thick annulus (radii 1 and 2, height 1; polar map r = 1 + xi1, angle pi xi2 / 4), "
               "viscosity 1")
        return (f"{name}: {dom}, TH IGA p={w['p']}, {n} elements, {op}, "
                f"P_D^G (geometry/viscosity-aware FD), {nrhs} seeded N(0,1) right-hand sides (pressure part "
                f"mean-free), MINRES tol 1e-8 from x0=0")
    return (f"{name}: {w['dim']}D unit {'cube' if w['dim'] == 3 else 'square'}, {w['disc']} IGA, pressure degree "
            f"p={w['p']}, {n} elements, {nrhs} seeded N(0,1) right-hand sides (pressure part mean-free), "
            f"tol 1e-8 from x0=0")


def peaks():
    try:
        return json.load(open(MEASURED_PEAKS))
    except (OSError, ValueError):
        return {}


def oracle_operator(w):
    """(S, matvec, preconditioner) of the oracle for a workload dict."""
    import synth
    from oracle import stokes
    knots = [synth.open_uniform_knots(n, w["p"]) for n in w["n_el"]]
    S = stokes.build(knots, w["p"], w.get("disc", "TH"))
    if w.get("geometry") in ("sine_bump", "annulus"):
        from oracle import geometry as geo
        G = geo.Grid(S, geometry_kind=w["geometry"])
        P = geo.PDG(S, G)
        return S, (lambda v: geo.matvec(S, G, v)), P.apply
    return S, (lambda v: stokes.matvec(S, v)), (lambda v: stokes.apply_PD_inv(S, v))


def cpu_oracle_sample(w, seeds, iters_per_solve, k_iters=2, op=None):
    """The oracle as it stands on the host cores: k_iters MINRES iterations at
    full workload size on one right-hand side, scaled to solves/s with the
    iteration count of a full solve (operator setup not timed)."""
    import synth
    from oracle import minres
    S, mv, pc = op if op is not None else oracle_operator(w)
    b = synth.rhs(seeds[0], S.block_sizes)
    t0 = time.perf_counter()
    minres.minres(mv, b, pc, tol=0.0, maxit=k_iters)
    dt = time.perf_counter() - t0
    t_iter = dt / (k_iters + 1)          # k iterations + the initial matvec/apply
    value = 1.0 / (t_iter * iters_per_solve)
    return dict(value=value, unit="solves/s", cores=os.cpu_count(), kind="oracle",
                sample=(f"{k_iters} MINRES iterations of the NumPy/SciPy FP64 oracle on 1 right-hand side at "
                        f"full size ({dt:.1f} s incl. the initial matvec+apply; operator setup untimed), "
                        f"per-iteration time x {iters_per_solve:.1f} iterations per solve; BLAS threads = default "
                        f"(all cores)"),
                seconds=dt, t_iter_s=t_iter)


def cpu_oracle_single_thread(workload_name, iters_per_solve, k_iters=1):
    """cpu_oracle_sample with one BLAS/OpenMP thread (the paper's setting: one
    core), in a child process started with those limits (they bind only before
    NumPy loads). The child execs a fresh interpreter and touches no GPU."""
    import subprocess
    import sys
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json, bench; w = bench.workload(%r); "
            "r = bench.cpu_oracle_sample(w, w['seeds'], %r, k_iters=%d); "
            "print(json.dumps({'value': r['value'], 'seconds': r['seconds']}))") % (
                workload_name, float(iters_per_solve), k_iters)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         cwd=os.path.dirname(os.path.abspath(__file__)), timeout=600)
    if out.returncode != 0:
        return {"unavailable": out.stderr.strip().splitlines()[-1] if out.stderr.strip() else "child failed"}
    r = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": r["value"], "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": (f"{k_iters} MINRES iteration(s) of the oracle on 1 right-hand side at full size with one "
                       f"BLAS thread ({r['seconds']:.1f} s incl. the initial matvec+apply), per-iteration time x "
                       f"{iters_per_solve:.1f} iterations per solve")}


def cpu_oracle_instances(specs, iters, k_iters=1, max_dof=4.0e6, count=3):
    """Oracle solves/s over a sample of independent instances: the first
    `count` instances with at most max_dof unknowns; each instance's solve time
    = its oracle per-iteration time x its iteration count."""
    import synth
    from oracle import minres
    picked, total, dts = [], 0.0, []
    for spec, it in zip(specs, iters):
        if len(picked) == count:
            break
        S, mv, pc = oracle_operator(spec)
        if S.n_total > max_dof:
            continue
        b = synth.rhs(spec.get("seed", 1), S.block_sizes)
        t0 = time.perf_counter()
        minres.minres(mv, b, pc, tol=0.0, maxit=k_iters)
        dt = time.perf_counter() - t0
        dts.append(dt)
        total += dt / (k_iters + 1) * it
        picked.append(f"{spec['dim']}D {spec.get('disc', 'TH')} p={spec['p']} n_el={tuple(spec['n_el'])}")
    value = len(picked) / total if total > 0 else None
    return dict(value=value, unit="solves/s", cores=os.cpu_count(), kind="oracle",
                sample=(f"{k_iters} oracle MINRES iteration(s) (+ initial matvec/apply) on each of {len(picked)} "
                        f"instances ({'; '.join(picked)}; the first with <= {max_dof:.0e} unknowns), solve time = "
                        f"per-iteration time x that instance's GPU iteration count; {sum(dts):.1f} s of CPU work"))


# ------------------------------------------------------------------ reference arm (oracle on CPU)

def oracle_full_solve(w, seed, op=None, maxit=2000):
    """One complete oracle P_D-MINRES solve (1 right-hand side, tol 1e-8, x0 = 0)
    on the host cores: (seconds, iterations)."""
    import synth
    from oracle import minres
    S, mv, pc = op if op is not None else oracle_operator(w)
    b = synth.rhs(seed, S.block_sizes)
    t0 = time.perf_counter()
    _, info = minres.minres(mv, b, pc, tol=1e-8, maxit=maxit, true_check=True)
    return time.perf_counter() - t0, int(info["iters"])


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.workload)
    kind = w.get("kind", "single")
    if kind in ("batched", "serving"):
        specs = instance_specs(args.workload, w)
        iters = 60.0
        vals, secs, cpu = [], [], None
        for k in range(args.warmup + args.steps):
            cpu = cpu_oracle_instances(specs, [iters] * len(specs), k_iters=1)
            if k >= args.warmup:
                vals.append(cpu["value"])
                secs.append(1.0 / cpu["value"])
        nrhs, cfg = 1, {"workload": args.workload + ": " + w_text(args.workload, w)}
        full = None
    else:
        op = oracle_operator(w)
        # the iteration count the per-iteration times are scaled by is the oracle's own, from one
        # complete solve of the first right-hand side (timed once, reported beside the steps)
        t_full, iters = oracle_full_solve(w, w["seeds"][0], op=op)
        full = {"seconds": t_full, "iterations": iters, "solves_per_s": 1.0 / t_full}
        vals, secs = [], []
        for k in range(args.warmup + args.steps):
            r = cpu_oracle_sample(w, w["seeds"], iters, k_iters=1, op=op)
            if k >= args.warmup:
                vals.append(r["value"])
                secs.append(r["t_iter_s"] * iters)
        nrhs, cfg = 1, {"workload": describe(args.workload, w, 1), "nrhs": 1}
        cpu = {"sample": "per step: 1 MINRES iteration (plus the initial matvec and apply) of the FP64 oracle at "
                         f"full size on 1 RHS, scaled by the {iters} iterations of the oracle's own complete "
                         f"solve of seed {w['seeds'][0]} (that solve: {t_full:.1f} s, timed once before the steps)"}
    value = statistics.median(vals)
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": cfg,
           "cpu_baseline": {"value": value, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": cpu["sample"]},
           "oracle_full_solve": full,
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def w_text(name, w):
    if w.get("kind") == "batched":
        return (f"{w['count']} independent unit-cube Taylor-Hood instances, p ~ U{{2..6}}, elements per direction "
                f"~ U{{16..96}} (draw seed {w['seed']}), one seeded N(0,1) right-hand side each "
                f"(seeds {w['rhs_seed0']}..{w['rhs_seed0'] + w['count'] - 1}), MINRES tol 1e-8 from x0=0")
    return (f"Poisson arrivals at rates {w['rates']} req/s, {w['per_rate']} requests per rate; 50/50 mix of 3D "
            f"unit-cube TH (p ~ U{{2..6}}, elements per direction ~ U{{16..96}}) and 2D TH/RT (p ~ U{{2..8}}, "
            f"elements per direction ~ U{{32..256}}); MINRES tol 1e-8")


def instance_specs(name, w):
    import synth
    if w.get("kind") == "batched":
        out = synth.batched_instances(w["seed"], w["count"])
        for i, o in enumerate(out):
            o["seed"] = w["rhs_seed0"] + i
        return out
    return synth.serving_requests(0, w["rates"][0], w["per_rate"], w["seed"], w["mix_seed"])


# ------------------------------------------------------------------ GPU arm

def run_gpu(args):
    import numpy as np
    import torch

    import paper_1712_00403_gb300 as fd
    import synth

    rep = Replicas("nccl")
    world, rank, local = rep.world, rep.rank, rep.local
    dev = torch.device("cuda", local)

    w = workload(args.workload)
    nrhs = args.nrhs or len(w["seeds"])
    if args.fd == "auto":
        # the mapped configuration names the split-BF16 form; the others split-TF32
        prec = fd.FD_BF16X6 if w.get("geometry") in ("sine_bump", "annulus") else fd.FD_TF32X3
    else:
        prec = {"f64": fd.FD_F64, "tf32": fd.FD_TF32X3, "bf16": fd.FD_BF16X6}[args.fd]
    knots = synth.knots_for(w)
    t_setup = time.perf_counter()
    mapped = w.get("geometry") in ("sine_bump", "annulus")
    mv = fd.MV_DF64 if args.matvec == "df64" else fd.MV_F64
    geo = dict(geometry=fd.GEOM_ANNULUS if w["geometry"] == "annulus" else fd.GEOM_SINE_BUMP,
               variant=fd.VARIANT_PD_GEO) if mapped else {}
    mfree = mapped and args.matrix_free
    if mfree:
        geo["matvec_form"] = fd.MATVEC_MATRIX_FREE
    P = fd.Stokes(knots, w["p"], disc=fd.TH if w["disc"] == "TH" else fd.RT, fd_precision=prec, max_rhs=nrhs,
                  matvec_precision=mv, **geo)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    # weak scaling: every rank solves its own batch (seeds shifted by rank)
    seeds = rep.seeds(w["seeds"], nrhs)
    B = np.stack([synth.rhs(s, P.block_sizes) for s in seeds])
    b = torch.tensor(B.reshape(-1), device=dev)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()

    gm = args.solver != "minres"
    gm_prec = fd.PREC_PC if args.solver == "gmres-pc" else fd.PREC_PT

    def solve_dev(bb, xx):
        if gm:
            return P.solve_gmres(bb, xx, prec=gm_prec, tol=1e-8, maxit=args.maxit, restart=args.restart,
                                 stream=stream)
        return P.solve(bb, xx, tol=1e-8, maxit=args.maxit, stream=stream)

    def step():
        x.zero_()
        return solve_dev(b, x)

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()
    rep.barrier()
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
    ms = rep.max(e0.elapsed_time(e1))
    clocks = clk.summary()
    total_solves = rep.sum(args.steps * nrhs)
    value = total_solves / (ms / 1e3)

    iters = [i["iterations"] for inf in infos for i in inf]
    iters_est = [i["iterations_estimate"] for inf in infos for i in inf]
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
                        max_rhs=1, **geo)
        s64 = torch.empty(P.n_total, dtype=torch.float64, device=dev)
        P64.apply_prec(b[:P.n_total].contiguous(), s64, stream=stream)
        torch.cuda.synchronize()
        apply_err = float(torch.linalg.norm(s[:P.n_total] - s64) / torch.linalg.norm(s64))
        P64.close()

    # roofline of the dominant kernel, timed live inside the timed region: for the matvec, CUDA events
    # around its compute launches alone (fdst_get_kernel_timing); for the FD apply, the preconditioner phase
    pk = peaks()
    per_mv = tm["ms_matvec"] / max(tm["n_matvec"], 1)
    per_pc = tm["ms_prec"] / max(tm["n_prec"], 1)
    k_ms = tm["ms_matvec_kernels"] / max(tm["n_matvec"], 1)          # compute launches per matvec
    k_launch_ms = tm["ms_matvec_kernels"] / max(tm["n_matvec_kernel_launches"], 1)
    unit = "TFLOP/s"
    if per_mv >= per_pc and mapped and not mfree:
        nnz = P.flops_matvec / 2.0
        kern = ("csr_spmv_%s (assembled mapped Stokes operator, one warp per row, 4 RHS per pass)"
                % ("df64" if mv == fd.MV_DF64 else "f64"))
        # algorithmic bytes per launch: values (8 B: FP64 or an FP32 pair) + column indices once,
        # row pointers once, x read and y written once per entry and RHS
        flops = None
        byts = 12.0 * nnz + 8.0 * (P.n_total + 1) + 16.0 * P.n_total * nrhs
        t_ms, launch_ms = k_ms, k_launch_ms
        peak, bound = pk.get("hbm_gbs", 6701.5), "hbm"
        peak_note = "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    elif per_mv >= per_pc and mv == fd.MV_F64:
        kern, flops, t_ms, launch_ms = ("k_band (FP64 banded Kronecker mode products of the matvec)",
                                        P.flops_matvec * nrhs, k_ms, k_launch_ms)
        peak = FP64_NOMINAL_TFLOPS
        peak_note = "FP64 DFMA nominal 1.25 TFLOP/s (recipe table; measured DFMA chain 1.20)"
        bound = "alu"
    elif per_mv >= per_pc:
        # double-float: 12 FP32 lane operations per banded multiply-add of the plan (exact product
        # with 1 FMUL + 3 FFMA, TwoSum and error accumulation with 8 FADD); the FP32 pipe issues one
        # lane operation per lane and clock whatever its kind, so the ceiling is the lane rate
        kern = ("k_band_df (double-float banded products of the sum-factorized mapped matvec: point-basis "
                "values/derivatives and their transposes; the point stage not counted)" if mfree else
                "k_band_df (double-float banded Kronecker mode products of the matvec)")
        flops, t_ms, launch_ms = P.flops_matvec / 2.0 * 12.0 * nrhs, k_ms, k_launch_ms
        peak, unit = FP32_LANE_TOPS, "Top/s"
        peak_note = ("FP32 lane operations: 152 SMs x 128 FP32 lanes x 2070 MHz = 40.3 T/s nominal "
                     "(an FFMA chain measured 37.5 T/s); achieved counts 12 per multiply-add of the plan")
        bound = "alu"
    else:
        kern, flops, t_ms = "k_gemm_tc (FD apply phase)", P.flops_apply * nrhs, per_pc
        launch_ms = per_pc
        if prec == fd.FD_F64:
            kern = "k_gemm_f64 (FD apply phase)"
            peak, bound = FP64_NOMINAL_TFLOPS, "alu"
            peak_note = "FP64 DFMA nominal 1.25 TFLOP/s (recipe table; measured DFMA chain 1.20)"
        elif prec == fd.FD_BF16X6:
            peak = pk.get("bf16_tflops_sustained", 1748.4)
            bound = "tensor"
            peak_note = "measured bf16 sustained (MEASURED_PEAKS.json)"
            flops *= 6  # six split products per contraction
        else:
            peak = pk.get("bf16_tflops_sustained", 1748.4) * TF32_OVER_BF16
            bound = "tensor"
            peak_note = "TF32 = measured bf16 sustained x nominal TF32/BF16 ratio"
            flops *= 3  # three split products per contraction
    if bound == "hbm":
        achieved, unit = byts / (t_ms / 1e3) / 1e9, "GB/s"
    else:
        achieved = flops / (t_ms / 1e3) / 1e12
    traffic, traffic_note = None, None
    if per_mv >= per_pc and mv == fd.MV_DF64 and not mfree:
        tr = MATVEC_TRAFFIC["k_spmv_df" if mapped else "k_band_df"]
        if tr["nrhs"] == nrhs:
            scale = (P.flops_matvec / 2.0) / tr["nnz"] if mapped else P.n_total / tr["entries"]
            # per launch, like achieved: a matvec's bytes over its launches
            traffic = tr["bytes"] * scale / tr["launches"]
            traffic_note = ("ncu DRAM bytes per launch (%s), %s" % (
                "one launch captured on the 16^3 mapped cube, scaled by nonzero count" if mapped else
                "mean of the %d launches of one matvec captured on 1,673,830 entries per RHS, scaled by "
                "entry count" % tr["launches"], "B"))
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": traffic, "traffic_note": traffic_note, "kernel": kern, "ms_per_launch": launch_ms,
                "ms_per_phase": t_ms, "peak_source": peak_note}

    # end to end through the host-pointer entry point (pinned host buffers); GMRES has no
    # host-pointer entry point, so its copies are made here around the device call
    bh = torch.empty(b.numel(), dtype=torch.float64, pin_memory=True)
    bh.copy_(b.cpu())
    xh = torch.zeros(b.numel(), dtype=torch.float64, pin_memory=True)
    bn, xn = bh.numpy(), xh.numpy()
    e2e_steps = max(2, args.steps // 3)
    if not gm:
        # untimed warm-up call: the host-pointer entry point allocates its device staging
        # buffers on first use
        P.solve_host(bn, xn, tol=1e-8, maxit=args.maxit, stream=stream, zero_guess=True)
    torch.cuda.synchronize()
    rep.barrier()
    e2e_each = []
    with ClockSampler(local) as e2e_clk:
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            t_one = time.perf_counter()
            if gm:
                bd = bh.to(dev, non_blocking=True)
                xd = torch.zeros_like(bd)
                solve_dev(bd, xd)
                xh.copy_(xd, non_blocking=True)
                torch.cuda.synchronize()
            else:
                # x0 = 0 cleared on the device: only b goes in, only the solutions come back
                P.solve_host(bn, xn, tol=1e-8, maxit=args.maxit, stream=stream, zero_guess=True)
            e2e_each.append(1e3 * (time.perf_counter() - t_one))
        e2e_s = time.perf_counter() - t0
    e2e = {"value": rep.job_rate(e2e_steps * nrhs, e2e_s), "unit": "solves/s",
           "h2d_bytes_per_step": b.numel() * 8, "d2h_bytes_per_step": b.numel() * 8,
           "ms_each_step": e2e_each, "clocks": e2e_clk.summary(),
           "entry": "fdst_solve_gmres with torch copies" if gm else "fdst_solve_host_zero (pinned host b in, x out)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not gm:
        mean_it = float(np.mean(iters))
        cpu = cpu_oracle_sample(w, w["seeds"], mean_it, k_iters=1 if mapped else 2)
        cpu.pop("seconds", None)
        cpu.pop("t_iter_s", None)
        cpu["sample"] += f" (the GPU solves' mean iteration count, {mean_it:.2f})"
        if not mapped:
            cpu["single_thread"] = cpu_oracle_single_thread(args.workload, mean_it)

    # the plain-FP64 form of the same solve (FD apply and matvec in FP64), same right-hand sides
    dev_bytes, flops_mv, n_tot = P.device_bytes, P.flops_matvec, P.n_total
    fp64 = None
    if not gm and not args.no_fp64 and not (prec == fd.FD_F64 and mv == fd.MV_F64):
        P.close()
        P = None
        fp64 = fp64_leg(args, w, knots, nrhs, b, stream, geo, rep)

    if rank == 0:
        dtype = {fd.FD_F64: "f64", fd.FD_TF32X3: "f64+tf32x3", fd.FD_BF16X6: "f64+bf16x6"}[prec]
        if mv == fd.MV_DF64:
            dtype += " (matvec df64)"
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": dtype, "data": "synthetic",
               "config": {"workload": describe(args.workload, w, nrhs, mfree), "nrhs_per_gpu": nrhs,
                          "device_bytes": dev_bytes,
                          "solver": ("P_D-MINRES" if not gm else "%s-GMRES (%s form, Krylov basis %d)" % (
                              "P_C" if args.solver == "gmres-pc" else "P_T",
                              "left" if prec == fd.FD_F64 else "flexible", args.restart)),
                          "fd_precision": {fd.FD_F64: "f64", fd.FD_TF32X3: "tf32x3", fd.FD_BF16X6: "bf16x6"}[prec],
                          "matvec": (("double-float (FP32 pairs, 48-bit significand) %s in the iterations; "
                                      "true residual in FP64") % (
                                          "sum-factorized matrix-free operator" if mfree else
                                          "CSR SpMV (%d nonzeros)" % int(flops_mv / 2)
                                          if mapped else "banded Kronecker products"))
                                    if mv == fd.MV_DF64 else
                                    ("FP64 CSR SpMV (%d nonzeros)" % int(flops_mv / 2) if mapped else "FP64"),
                          "n_total": n_tot,
                          "l2": "inputs larger than L2 (each step streams %d x %.0f MB vectors)" % (
                              nrhs, n_tot * 8 / 1e6),
                          "parallelism": rep.parallelism},
               ("gmres" if gm else "minres"): {
                   "iterations_min": min(iters), "iterations_max": max(iters), "status": statuses,
                   "true_rel_res_max": true_res,
                   "iterations_estimate_min": min(iters_est), "iterations_estimate_max": max(iters_est)},
               "fd_apply": {"applies_per_s": applies_per_s, "gdof_per_s": applies_per_s * n_tot / 1e9,
                            "ms_per_batch": ms_apply, "rel_err_vs_f64": apply_err},
               "phases_ms_per_iter": None if gm else {"matvec": per_mv, "prec": per_pc,
                                                      "vector": tm["ms_vector"] / max(tm["n_matvec"], 1)},
               "setup_s": t_setup, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "clocks": clocks}
        if fp64 is not None:
            out["fp64"] = fp64
        print(json.dumps(out), flush=True)
    if P is not None:
        P.close()
    rep.close()


def fp64_leg(args, w, knots, nrhs, b, stream, geo, rep):
    """The same solve with the FD apply and the matvec in plain FP64 (the paper's
    precision): one warm-up solve step, then args.fp64_steps timed steps on the
    launching stream; plus the FP64 FD apply alone."""
    import torch

    import paper_1712_00403_gb300 as fd
    P = fd.Stokes(knots, w["p"], disc=fd.TH if w["disc"] == "TH" else fd.RT, fd_precision=fd.FD_F64,
                  max_rhs=nrhs, matvec_precision=fd.MV_F64, **geo)
    x = torch.zeros_like(b)
    x.zero_()
    P.solve(b, x, tol=1e-8, maxit=args.maxit, stream=stream)
    torch.cuda.synchronize()
    rep.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for _ in range(args.fp64_steps):
        x.zero_()
        infos.append(P.solve(b, x, tol=1e-8, maxit=args.maxit, stream=stream))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = rep.max(e0.elapsed_time(e1))
    s = torch.empty_like(b)
    P.apply_prec(b, s, stream=stream)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(3):
        P.apply_prec(b, s, stream=stream)
    a1.record(stream)
    torch.cuda.synchronize()
    ms_apply = a0.elapsed_time(a1) / 3
    its = [i["iterations"] for inf in infos for i in inf]
    out = {"value": rep.sum(args.fp64_steps * nrhs) / (ms / 1e3), "unit": "solves/s", "steps": args.fp64_steps,
           "warmup": 1, "ms_per_step": ms / args.fp64_steps, "dtype": "f64", "fd_precision": "f64", "matvec": "FP64",
           "minres": {"iterations_min": min(its), "iterations_max": max(its),
                      "status": sorted(set(i["status"] for inf in infos for i in inf)),
                      "true_rel_res_max": max(i["true_rel_res"] for inf in infos for i in inf)},
           "fd_apply": {"ms_per_batch": ms_apply, "applies_per_s": nrhs / (ms_apply / 1e3),
                        "gdof_per_s": nrhs / (ms_apply / 1e3) * P.n_total / 1e9},
           "note": "same right-hand sides and stopping rule; warm-up: one full solve step"}
    P.close()
    return out


# ------------------------------------------------------------------ batched workload

def _make_handles(fd, specs, local, threads=8, **kw):
    """Set up one device handle per instance on host threads (the library's
    setup is thread-safe; each thread selects the rank's GPU)."""
    import torch
    from concurrent.futures import ThreadPoolExecutor

    import synth

    def one(spec):
        torch.cuda.set_device(local)
        knots = [synth.open_uniform_knots(n, spec["p"]) for n in spec["n_el"]]
        return fd.Stokes(knots, spec["p"], disc=fd.TH if spec.get("disc", "TH") == "TH" else fd.RT, max_rhs=1, **kw)

    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(one, specs))


def run_batched(args):
    import numpy as np
    import torch

    import paper_1712_00403_gb300 as fd
    import synth

    rep = Replicas("nccl")
    world, rank, local = rep.world, rep.rank, rep.local
    dev = torch.device("cuda", local)
    w = workload(args.workload)
    specs = instance_specs(args.workload, w)
    for s_ in specs:
        s_["seed"] = rep.seed(s_["seed"])
    stream = torch.cuda.current_stream()

    def timed_batch(prec, steps, warmup, host_e2e=False):
        t0 = time.perf_counter()
        hs = _make_handles(fd, specs, local, fd_precision=prec, matvec_precision=fd.MV_DF64)
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        B = fd.Batch(hs, autotune=True)
        t_tune = time.perf_counter() - t0
        bs = [torch.tensor(synth.rhs(sp["seed"], h.block_sizes), device=dev) for sp, h in zip(specs, hs)]
        xs = [torch.zeros_like(b) for b in bs]

        def step():
            for x in xs:
                x.zero_()
            return B.solve(bs, xs, tol=1e-8, maxit=args.maxit, stream=stream)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        rep.barrier()
        l0 = fd.kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(steps):
                infos.append(step())
            e1.record(stream)
            torch.cuda.synchronize()
        launches = fd.kernel_launches() - l0
        ms = rep.max(e0.elapsed_time(e1))
        res = dict(ms=ms, infos=infos, launches=launches, clocks=clk.summary(), setup_s=t_setup, tune_s=t_tune,
                   info=B.info(), n_total=[h.n_total for h in hs])
        if host_e2e:
            # end to end: pinned host right-hand sides in, solutions out, copies inside the timed region
            bh = [torch.empty(b.numel(), dtype=torch.float64, pin_memory=True).copy_(b.cpu()) for b in bs]
            xh = [torch.empty(b.numel(), dtype=torch.float64, pin_memory=True) for b in bs]
            torch.cuda.synchronize()
            rep.barrier()
            t0 = time.perf_counter()
            for b, bhost in zip(bs, bh):
                b.copy_(bhost, non_blocking=True)
            step()
            for x, xhost in zip(xs, xh):
                xhost.copy_(x, non_blocking=True)
            torch.cuda.synchronize()
            res["e2e_s"] = time.perf_counter() - t0
            res["bytes"] = sum(b.numel() for b in bs) * 8
        # FD apply error vs the FP64 apply on a sample of instances (kept for the FP64 pass)
        res["apply_out"] = []
        for i in range(4):
            s_out = torch.empty_like(bs[i])
            hs[i].apply_prec(bs[i], s_out, stream=stream)
            res["apply_out"].append(s_out)
        torch.cuda.synchronize()
        B.close()
        for h in hs:
            h.close()
        return res

    tc = timed_batch(fd.FD_TF32X3, args.steps, args.warmup, host_e2e=True)
    f64 = None if args.no_fp64 else timed_batch(fd.FD_F64, max(1, args.steps // 3 or 1), max(3, args.warmup // 2))
    errs = ([float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(tc["apply_out"], f64["apply_out"])]
            if f64 else None)
    n = len(specs)
    value = rep.sum(args.steps * n) / (tc["ms"] / 1e3)
    e2e_value = rep.job_rate(n, tc["e2e_s"])
    it_tc = [i["iterations"] for inf in tc["infos"] for i in inf]
    it_64 = [i["iterations"] for inf in f64["infos"] for i in inf] if f64 else []
    st_tc = sorted(set(i["status"] for inf in tc["infos"] for i in inf))
    tr_tc = max(i["true_rel_res"] for inf in tc["infos"] for i in inf)
    tr_64 = max(i["true_rel_res"] for inf in f64["infos"] for i in inf) if f64 else None
    value64 = rep.sum(len(f64["infos"]) * n) / (f64["ms"] / 1e3) if f64 else None
    # roofline of the grouped split-TF32 FD apply (one launch chain over all instances, autotuner timing)
    flops_apply = 0.0
    for sp in specs:
        p = sp["p"]
        nv = [2 * e + p - 2 for e in sp["n_el"]]
        nq = [e + p for e in sp["n_el"]]
        Nv, Nq = float(np.prod(nv)), float(np.prod(nq))
        flops_apply += 3 * 4 * Nv * sum(nv) + 4 * Nq * sum(nq)
    pk = peaks()
    peak = pk.get("bf16_tflops_sustained", 1748.4) * TF32_OVER_BF16
    ms_apply = tc["info"]["ms_apply"]
    achieved = 3 * flops_apply / (ms_apply / 1e3) / 1e12 if ms_apply > 0 else None
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "kernel": "grouped split-TF32 FD apply over all 64 instances (tcgen05), autotuner's CUDA-event time",
                "ms_per_launch": ms_apply,
                "peak_source": "TF32 = measured bf16 sustained x nominal TF32/BF16 ratio; flops = 3 split products "
                               "x 4 N sum(n_d) per velocity component + 4 N_q sum(n_q) per pressure"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_instances(specs, it_tc[:n], k_iters=1)
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": tc["ms"] / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64+tf32x3 (matvec df64)", "data": "synthetic",
               "config": {"workload": args.workload + ": " + w_text(args.workload, w),
                          "total_dof": int(sum(tc["n_total"])), "max_dof": int(max(tc["n_total"])),
                          "l2": "inputs larger than L2 (%.1f GB of right-hand sides)" % (sum(tc["n_total"]) * 8e-9),
                          "parallelism": rep.parallelism},
               "minres": {"iterations_min": min(it_tc), "iterations_max": max(it_tc), "iterations_mean":
                          float(np.mean(it_tc)), "status": st_tc, "true_rel_res_max": tr_tc,
                          "iterations_estimate_mean": float(np.mean([i["iterations_estimate"] for inf in tc["infos"]
                                                                      for i in inf]))},
               "fp64_fd": ({"solves_per_s": value64, "ms_per_step": f64["ms"] / len(f64["infos"]),
                            "iterations_mean": float(np.mean(it_64)), "true_rel_res_max": tr_64,
                            "ms_apply_grouped": f64["info"]["ms_apply"],
                            "iteration_delta_max": max(abs(a - b) for a, b in zip(it_tc[:n], it_64[:n]))}
                           if f64 else None),
               "fd_apply_rel_err_vs_f64": errs,
               "autotune": tc["info"], "setup_s": tc["setup_s"], "autotune_s": tc["tune_s"],
               "roofline": roofline, "cpu_baseline": cpu,
               "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": tc["bytes"],
                       "d2h_bytes_per_step": tc["bytes"]},
               "gpu_launches": tc["launches"], "clocks": tc["clocks"]}
        print(json.dumps(out), flush=True)
    rep.close()


# ------------------------------------------------------------------ serving workload

def run_serving(args):
    import numpy as np
    import torch

    import paper_1712_00403_gb300 as fd
    import synth

    rep = Replicas("nccl")
    world, rank, local = rep.world, rep.rank, rep.local
    w = workload(args.workload)

    def stream_of(reqs):
        out = []
        for r in reqs:
            knots = [synth.open_uniform_knots(n, r["p"]) for n in r["n_el"]]
            sizes = block_sizes(r)
            out.append((r, knots, synth.rhs(rep.seed(r["seed"]), sizes)))
        return out

    def serve(reqs, max_active=args.serving_max_active, fd_precision=fd.FD_TF32X3, matvec_precision=fd.MV_DF64):
        server = fd.Server(max_active=max_active, iters_per_step=args.serving_iters, fd_precision=fd_precision,
                           matvec_precision=matvec_precision, tol=1e-8, maxit=args.maxit)
        ids, k = [], 0
        l0 = fd.kernel_launches()
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while k < len(reqs) and reqs[k][0]["t"] <= now:
                r, knots, b = reqs[k]
                ids.append(server.submit(knots, r["p"], b, r["t"], disc=fd.TH if r["disc"] == "TH" else fd.RT))
                k += 1
            active, queued, finished = server.step(time.perf_counter() - t0)
            if finished == len(reqs):
                break
            if active == 0 and queued == 0 and k < len(reqs):
                time.sleep(max(0.0, reqs[k][0]["t"] - (time.perf_counter() - t0)))
        t_end = time.perf_counter() - t0
        launches = fd.kernel_launches() - l0
        results = [server.result(i) for i in ids]
        st = server.stats()
        server.close()
        return results, t_end, launches, st

    # warm-up: a short stream of other requests (context, kernels, autotuning paths)
    warm = stream_of(synth.serving_requests(9, 200.0, 8, w["seed"] + 90, w["mix_seed"] + 90, nel3=(8, 16)))
    for _ in range(max(1, args.warmup // 3)):
        serve(warm)
    per_rate, all_lat, total_solves, total_time, launches, clocks = [], [], 0, 0.0, 0, None
    checked = []   # served solutions that the cpu_baseline leg checks against the oracle
    with ClockSampler(local) as clk:
        for ri, rate in enumerate(w["rates"]):
            reqs = stream_of(synth.serving_requests(ri, rate, w["per_rate"], w["seed"], w["mix_seed"],
                                                    nel3=(16, args.serving_nel3_max)))
            torch.cuda.synchronize()
            res, t_end, nl, st = serve(reqs)
            launches += nl
            lat = [r["t_done"] - r["t_arrival"] for r in res]
            wait = [r["t_admit"] - r["t_arrival"] for r in res]
            ok = sum(r["status"] == "OK" for r in res)
            thr = len(res) / (t_end - reqs[0][0]["t"])
            per_rate.append({"rate_req_s": rate, "requests": len(res), "ok": ok, "solves_per_s": thr,
                             "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                             "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                             "mean_admission_wait_ms": 1e3 * float(np.mean(wait)),
                             "true_rel_res_max": max(r["true_rel_res"] for r in res),
                             "iterations_mean": float(np.mean([r["iterations"] for r in res])),
                             "handles_created": st["handles_created"], "handles_reused": st["handles_reused"],
                             "max_active_seen": st["max_active_seen"]})
            all_lat += lat
            total_solves += len(res)
            total_time += t_end - reqs[0][0]["t"]
            # kept for the cpu_baseline leg: the three smallest requests of each stream
            if rank == 0 and world == 1 and not args.no_cpu_baseline:
                order = sorted(range(len(reqs)), key=lambda i: int(np.sum(block_sizes(reqs[i][0]))))
                for j, i in enumerate(order[:3]):
                    checked.append((reqs[i], res[i], ri == 0 and j == 0))
        clocks = clk.summary()
    tot = [rep.sum(total_solves), rep.max(total_time)]
    value = tot[0] / tot[1]
    # the plain-FP64 form (FD apply and matvec in FP64) served on the first rate's stream, untimed by the
    # headline value above, beside it for comparison
    fp64 = None
    if not args.no_fp64:
        reqs = stream_of(synth.serving_requests(0, w["rates"][0], w["per_rate"], w["seed"], w["mix_seed"],
                                                nel3=(16, args.serving_nel3_max)))
        torch.cuda.synchronize()
        res, t_end, _, st = serve(reqs, fd_precision=fd.FD_F64, matvec_precision=fd.MV_F64)
        lat = [r["t_done"] - r["t_arrival"] for r in res]
        fp64 = {"rate_req_s": w["rates"][0], "requests": len(res), "ok": sum(r["status"] == "OK" for r in res),
                "solves_per_s": len(res) / (t_end - reqs[0][0]["t"]),
                "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "true_rel_res_max": max(r["true_rel_res"] for r in res),
                "iterations_mean": float(np.mean([r["iterations"] for r in res])),
                "note": "same stream as the first rate of the mixed run, FD apply and matvec in FP64"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        specs = [r for r, _, _ in stream_of(synth.serving_requests(0, w["rates"][0], w["per_rate"], w["seed"],
                                                                  w["mix_seed"], nel3=(16, args.serving_nel3_max)))]
        its = [pr["iterations_mean"] for pr in per_rate[:1]] * len(specs)
        cpu = cpu_oracle_instances(specs, its, k_iters=1)
        cpu["sample"] += "; iteration count = mean GPU iterations of the 50 req/s stream"
        # per-request error vs the FP64 oracle (after every timed region): true residual under the
        # oracle operator, and distance to the oracle's own solve for the smallest of the first stream
        cpu["per_request_error_vs_fp64_oracle"] = [oracle_error(rq, rs, solve=sv) for rq, rs, sv in checked]
    if rank == 0:
        h2d = int(sum(np.sum(block_sizes(r)) for r in
                      synth.serving_requests(0, w["rates"][0], w["per_rate"], w["seed"], w["mix_seed"],
                                             nel3=(16, args.serving_nel3_max))) * 8)
        out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
               "steps": len(w["rates"]), "warmup": max(1, args.warmup // 3),
               "ms_per_step": 1e3 * float(tot[1]) / len(w["rates"]), "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64+tf32x3 (matvec df64)", "data": "synthetic",
               "config": {"workload": "serving: " + w_text(args.workload, w),
                          "server": "max_active %d, %d MINRES iterations per scheduler step, HBM budget 90%% of "
                                    "free, handles set up on 8 host threads" % (args.serving_max_active,
                                                                                args.serving_iters),
                          "timing": "host wall clock from each stream's first arrival to its last completion "
                                    "(latency = completion - arrival, host clock)",
                          "parallelism": rep.parallelism},
               "serving": {"per_rate": per_rate, "p50_ms_all": 1e3 * float(np.percentile(all_lat, 50)),
                           "p99_ms_all": 1e3 * float(np.percentile(all_lat, 99))},
               "cpu_baseline": cpu,
               "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
                       "note": "requests enter and leave as host arrays; the value above is already end to end"},
               "roofline": None, "gpu_launches": launches, "clocks": clocks}
        if fp64 is not None:
            out["fp64"] = fp64
        print(json.dumps(out), flush=True)
    rep.close()


def block_sizes(r):
    p = r["p"]
    n_el = r["n_el"]
    if r.get("disc", "TH") == "TH":
        nv = int(np.prod([2 * e + p - 2 for e in n_el]))
        return [nv] * len(n_el) + [int(np.prod([e + p for e in n_el]))]
    out = []
    for k in range(len(n_el)):
        out.append(int(np.prod([(e + p - 1) if d == k else (e + p) for d, e in enumerate(n_el)])))
    return out + [int(np.prod([e + p for e in n_el]))]


def oracle_error(req, res, solve=False):
    """True relative residual of a served solution under the oracle's FP64
    operator and, with solve=True, its distance to the oracle's own MINRES
    solution (tolerance 1e-10)."""
    from oracle import minres
    r, knots, b = req
    S, mv, pc = oracle_operator(r)
    x = res["x"]
    out = {"request": f"{r['dim']}D {r['disc']} p={r['p']} n_el={tuple(r['n_el'])}", "n": int(S.n_total),
           "oracle_rel_res": float(np.linalg.norm(b - mv(x)) / np.linalg.norm(b))}
    if solve:
        xo, _ = minres.minres(mv, b, pc, tol=1e-10, maxit=2000, true_check=True)
        out["rel_err_vs_oracle_solve"] = float(np.linalg.norm(x - xo) / np.linalg.norm(xo))
    return out


def main():
    args = parse()
    kind = workload(args.workload).get("kind", "single")
    if args.impl == "reference":
        run_reference(args)
    elif kind == "batched":
        run_batched(args)
    elif kind == "serving":
        run_serving(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
