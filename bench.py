"""Benchmark: MLMC time-to-RMSE of the mixed-precision MPML estimator on one GB300.

Workload (one "step"): the whole hot path of one adaptive MLMC estimate --
Philox draws, tensor-core KL synthesis, every fine and coarse solve of every
level in resident-solve launches (FP32 inner CG preconditioned by a multigrid
V-cycle, a 16-bit-stored coefficient on coarse levels, FP64 iterative
refinement to the per-level accuracy of Eq. (4.12)), QoI and level statistics,
and the N_l updates of Alg. 4.1 -- on the five-level hierarchy h = 1/16 .. 1/256
with a 64-term KL field (exponential covariance, sigma^2 = 1, correlation
length 0.3), f = 1, Q = int u, N_init = 100 on every level, target RMSE 1e-3.

value    = seconds per estimate (device time between CUDA events on the stream).
e2e      = the same through the C ABI from host data, on a context set up once
           (its creation, which builds and uploads the basis tables, is reported
           as context_create_s): the step's seed set, the estimate, the result on
           the host.
roofline = the resident solve kernel: algorithmic bytes / event time of its
           launches (each on its own stream), against the measured HBM copy
           bandwidth; share_of_step = union of those launches on the device
           timeline / step time.
fp64     = the two FP64 forms (fixed 1e-10 and adaptive delta_l) on the same
           workload, seeds, --steps and --warmup.
cfg3_sweep / cfg4_adjoint / cfg5_7level = the other configurations, each on
           the same --steps and --warmup: the single-level sweep (4096 systems
           at n = 512, K = 128, four inner precisions), the adjoint gradients
           (1024 samples at n = 256, K = 256, box QoI) and the seven-level
           estimate (h = 1/16 .. 1/1024, K = 256, sigma^2 = 1.5, RMSE 2e-4).
cpu_baseline / --impl reference = the CPU FP64 oracle (banded Cholesky per
           solve) running the same Alg. 4.1 estimate in full, on the same seed,
           with one worker process per host core.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLMC time-to-RMSE (s) & solved DOF/s: mixed vs FP64 on 1 GB300; HBM GB/s"
WORKLOAD = dict(n0=16, m=2, L_max=4, kind=0, K=64, sigma2=1.0, corr_len=0.3, q=2.0, qoi=0, f=1.0)
TOL, N_INIT = 1e-3, 100
SEED = 1000          # Philox key of the timed estimate (rank r uses SEED + r)
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) per resident_solve launch of one timed step of this workload, averaged
# over the step's launches, from one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum
# (summary under profiles/; taken with the library's fixed launch settings, since under ncu the
# autotuner times serialised trials and picks other ones).  None whenever the solve kernel or its
# launch shape has changed since that capture.
SOLVE_TRAFFIC_BYTES_PER_LAUNCH = 7.38e9


DESC = ("mixed-precision batched MLMC: 5 levels h=1/16..1/256, KL 64 terms (exp. covariance sigma^2=1, "
        "corr length 0.3), f=1, Q=int u; FP32 inner CG preconditioned by a geometric multigrid V-cycle "
        "(FP16-stored coefficient while delta_l>=1e-4) with FP64 iterative refinement to delta_l of Eq. (4.12), "
        "k_p=0.05; N_init=100 per level, N_l from the optimal formula for RMSE 1e-3")
# The 7-level hierarchy (bench.py --case mlmc7): h = 1/16 .. 1/1024, K = 256, sigma^2 = 1.5, corr 0.1.
WORKLOAD7 = dict(n0=16, m=2, L_max=6, kind=0, K=256, sigma2=1.5, corr_len=0.1, q=2.0, qoi=0, f=1.0)
TOL7 = 2e-4
DESC7 = ("mixed-precision batched MLMC: 7 levels h=1/16..1/1024, KL 256 terms (exp. covariance sigma^2=1.5, "
         "corr length 0.1), f=1, Q=int u; FP32 inner CG preconditioned by a geometric multigrid V-cycle "
         "(FP16-stored coefficient while delta_l>=1e-4) with FP64 iterative refinement to delta_l of Eq. (4.12), "
         "k_p=0.05, FP64 re-runs of refinements that stagnate; N_init=100 per level, N_l from the optimal formula "
         "for RMSE 2e-4")


def workload_desc():
    return DESC


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle (only the cpu_baseline leg and --impl reference run this)
_ORACLE = {}


def _oracle_chunk(args):
    """Y = Q_l - Q_{l-1} of samples [first, first + count) of one level, by the oracle's FP64 solves."""
    wl, seed, level, first, count = args
    key = (tuple(sorted(wl.items())), seed)
    if key not in _ORACLE:
        sys.path.insert(0, ROOT)
        from oracle import mlmc as o_mlmc
        _ORACLE[key] = o_mlmc.Problem(n0=wl["n0"], m=wl["m"], L_max=wl["L_max"], field_kind=wl["kind"], K=wl["K"],
                                      sigma2=wl["sigma2"], corr_len=wl["corr_len"], q=wl["q"], seed=seed)
    Qf, Qc = _ORACLE[key].level_samples(level, first, count)
    return list(Qf - Qc)


def oracle_pool(procs):
    import multiprocessing as mp
    # one BLAS/OpenMP thread per worker: `procs` workers use `procs` cores (the children read this
    # environment when they import numpy)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        os.environ[var] = "1"
    return mp.get_context("spawn").Pool(procs)


def oracle_estimate(pool, procs, wl, tol, seed):
    """Alg. 4.1 of the oracle on the bench hierarchy (L fixed at L_max, N_init per level), its level
    samples evaluated in parallel chunks; returns (wall seconds, result dict)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle import mlmc as o_mlmc
    P = o_mlmc.Problem(n0=wl["n0"], m=wl["m"], L_max=wl["L_max"], field_kind=wl["kind"], K=wl["K"],
                       sigma2=wl["sigma2"], corr_len=wl["corr_len"], q=wl["q"], seed=seed)

    def sampler(level, first, count, deltas):
        nchunk = max(1, min(count, 4 * procs))
        bounds = [first + (count * c) // nchunk for c in range(nchunk + 1)]
        jobs = [(wl, seed, level, bounds[c], bounds[c + 1] - bounds[c]) for c in range(nchunk)
                if bounds[c + 1] > bounds[c]]
        return np.concatenate([np.asarray(y) for y in pool.map(_oracle_chunk, jobs)])

    t0 = time.perf_counter()
    res = o_mlmc.estimate(P, tol, N_init=N_INIT, L_start=wl["L_max"], sampler=sampler)
    return time.perf_counter() - t0, res


def oracle_warm(pool, procs, wl, seed):
    pool.map(_oracle_chunk, [(wl, seed, wl["L_max"], 10_000_000 + i, 1) for i in range(procs)])


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    procs = min(64, os.cpu_count() or 1)
    pool = oracle_pool(procs)
    try:
        oracle_warm(pool, procs, WORKLOAD, SEED)
        times, res = [], None
        for it in range(args.warmup + args.steps):
            secs, res = oracle_estimate(pool, procs, WORKLOAD, TOL, SEED)
            if it >= args.warmup:
                times.append(secs)
    finally:
        pool.close()
        pool.join()
    val = sum(times) / len(times)
    N = [int(x) for x in res["N"]]
    line = {"metric": METRIC, "value": val, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": val * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_desc(), "seed": SEED},
            "N_l": N, "estimate": float(res["estimate"]), "rmse": float(res["rmse"]),
            "cpu_baseline": {"value": val, "unit": "s", "cores": procs, "kind": "oracle",
                             "sample": "the whole estimate per step (Alg. 4.1 on the fixed 5-level hierarchy, "
                                       "N_l = %s, every fine and coarse solve by FP64 banded Cholesky), "
                                       "%d worker processes" % (N, procs)},
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libmlmc", choices=["libmlmc", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the library's fixed launch rules instead of the autotuner's choices")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the headline workload only (no 7-level, sweep and adjoint keys)")
    ap.add_argument("--case", default="mlmc",
                    choices=["mlmc", "mlmc7", "paper", "fixed3", "solve-l4", "kl-synth", "sweep", "adjoint"],
                    help="solve-l4: only the finest level's batch (100 samples, n = 256) of the workload: "
                         "field synthesis and one resident-solve launch per step; kl-synth: tensor-core "
                         "KL synthesis alone at the single-level sweep shapes (n = 512, K = 128, corr 0.1)")
    ap.add_argument("--kl-samples", type=int, default=4096)
    ap.add_argument("--kl-pitch-align", type=int, default=32,
                    help="kl-synth: the padded rows' pitch is (n+1)^2 rounded up to a multiple of this (elements)")
    ap.add_argument("--kl-pitch", type=int, default=0,
                    help="kl-synth: explicit pitch of the padded rows (elements; 0: from --kl-pitch-align)")
    ap.add_argument("--paper-runs", type=int, default=10, help="paper: seeds averaged per tolerance and form")
    ap.add_argument("--kl-prec", default="FP32", choices=["FP32", "FP64TC"],
                    help="kl-synth: output of the tensor-core synthesis")
    ap.add_argument("--sweep-samples", type=int, default=4096,
                    help="sweep: systems per batch (n = 512, K = 128, corr 0.1, fixed delta 1e-6)")
    ap.add_argument("--sweep-delta", type=float, default=1e-6,
                    help="sweep: relative residual (1e-6 for the measurement; larger for short profiles)")
    ap.add_argument("--prec", default="FP32", choices=["FP64", "FP32", "BF16S", "FP16S"],
                    help="sweep: inner precision (FP64 uses an FP64 field and FP64 vectors)")
    ap.add_argument("--pc", default="mg", choices=["mg", "jacobi"],
                    help="preconditioner of the CG inner solves")
    ap.add_argument("--mg-nu", type=int, default=0, help="multigrid smoothing sweeps (0: default)")
    ap.add_argument("--mg-coarse", type=int, default=0, help="multigrid coarsest-grid sweeps (0: default)")
    ap.add_argument("--mg-min", type=int, default=0, help="multigrid: halve grids while the half has at least "
                                                          "this many cells (0: default)")
    ap.add_argument("--tau-min", type=float, default=0.0,
                    help="solve-l4 and sweep: floor of the inner tolerance (0: per-precision default)")
    ap.add_argument("--med-items", type=int, default=0,
                    help="mlmc cases: most chunks of a system solved by a 128-thread group (0: the library's per-launch choice)")
    ap.add_argument("--ring", type=int, default=-1,
                    help="solve-l4: row-pipeline slots of the large CG solves (-1 automatic, 0 plain loads)")
    args = ap.parse_args()
    if args.case == "mlmc7":
        global WORKLOAD, TOL, DESC
        WORKLOAD, TOL, DESC = WORKLOAD7, TOL7, DESC7
        args.no_cpu_baseline = True     # the oracle's banded solves at h = 1/1024 take minutes per sample
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_05533_gb300 as M

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hbm_peak, _, peak_src = peaks()

    def opts(wl=None, tol=None, form=M.MLMC_FORM_MIXED):
        wl, tol = wl or WORKLOAD, tol or TOL
        o = M.mlmc_default_options()
        o.tol, o.L_start, o.N_init, o.form = tol, wl["L_max"], N_INIT, form
        o.fixed_delta = 1e-10
        return o

    def problem(seed):
        return M.make_problem(seed=seed, **WORKLOAD)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    if args.case == "solve-l4":
        return solve_l4_case(M, torch, dev, args, problem(SEED), hbm_peak, peak_src, flush, stream)
    if args.case == "kl-synth":
        return kl_synth_case(M, torch, dev, args, hbm_peak, peak_src, flush, stream)
    if args.case == "sweep":
        print(json.dumps(sweep_case(M, torch, dev, args, hbm_peak, peak_src, flush, stream)))
        return 0
    if args.case == "adjoint":
        print(json.dumps(adjoint_case(M, torch, dev, args, hbm_peak, peak_src, flush, stream)))
        return 0
    if args.case == "paper":
        print(json.dumps(paper_case(M, torch, dev, args, flush, stream)))
        return 0
    if args.case == "fixed3":
        return fixed3_case(M, torch, dev, args, flush, stream)

    def timed_runs(wl, tol, form, steps, warmup, seed0, profile=False):
        h = M.mlmc_create(M.make_problem(seed=seed0, **wl), local)
        try:
            if args.mg_nu or args.mg_coarse or args.pc != "mg":
                M.mlmc_set_precond(h, M.MLMC_PC_MG if args.pc == "mg" else M.MLMC_PC_JACOBI, args.mg_nu,
                                   args.mg_coarse)
            if args.med_items:
                M.mlmc_debug_set_medium_items(h, args.med_items)
            # launch settings: the autotuner times candidates on the warm-up estimates' launches
            M.mlmc_set_autotune(h, not args.no_autotune)
            if profile:
                M.mlmc_profile_enable(h, True)
            for w in range(warmup):
                M.mlmc_estimate(h, opts(wl, tol, form))
            tune = [M.mlmc_autotune_entry(h, i) for i in range(M.mlmc_autotune_count(h))]
            torch.cuda.synchronize()
            if profile:
                M.mlmc_profile_reset(h)
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            l0 = M.mlmc_launch_count()
            ms, results = [], []
            for s in range(steps):
                flush.fill_(float(s))                      # L2 flush between timed steps (outside the events)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = M.mlmc_estimate(h, opts(wl, tol, form))
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
                results.append(M.result_dict(res))
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            launches = M.mlmc_launch_count() - l0
            prof = M.mlmc_profile_get(h) if profile else None
            if prof is not None:
                prof["autotune"] = [{k: e[k] for k in ("shape", "med_items", "ring", "nu", "mg_min", "mg_coarse", "mg_omega", "mg_smem", "theta",
                                                        "tau_min", "best_ms", "default_ms", "trials")} for e in tune]
        finally:
            M.mlmc_destroy(h)
        return ms, results, launches, prof

    def fp64_forms(wl, tol):
        """The plain FP64 MLMC (fixed 1e-10) and FP64 with the adaptive delta_l, same workload, seeds,
        steps and warm-up as the mixed form."""
        out = {}
        for name, form in (("fp64_fixed_1e-10", M.MLMC_FORM_FP64_FIXED), ("fp64_adaptive", M.MLMC_FORM_FP64_ADAPTIVE)):
            fms, fres, _, _ = timed_runs(wl, tol, form, args.steps, args.warmup, SEED + rank)
            out[name] = {"seconds": sum(fms) / len(fms) / 1e3, "steps": len(fms), "N_l": fres[-1]["N"],
                         "inner_iters": sum(fres[-1]["inner_iters"]), "estimate": fres[-1]["estimate"],
                         "rmse": fres[-1]["rmse"]}
        return out

    with ClockSampler(local) as clk:
        ms, results, launches, prof = timed_runs(WORKLOAD, TOL, M.MLMC_FORM_MIXED, args.steps, args.warmup,
                                                 SEED + rank, True)
    total_ms = sum(ms)
    if dist:
        from paper_2503_05533_gb300 import replicas
        total_ms = replicas.max_over_ranks(dist, total_ms, device=dev)
    ms_per_step = total_ms / args.steps
    dofs = sum(sum(r["dofs"]) for r in results) / len(results)
    iters = [sum(r["inner_iters"]) for r in results]

    fp64 = {} if args.no_fp64 else fp64_forms(WORKLOAD, TOL)

    # e2e through the C ABI from host data: the step's input (a new seed) set on the host, the estimate,
    # its result read back; the context (KL basis tables built on the host and uploaded, workspaces) is
    # set up once, like a model loaded before serving, and its cost is reported beside (context_create_s)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = M.mlmc_create(problem(2000), local)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    e2e_s, h2d, d2h = [], 0, 0
    try:
        M.mlmc_set_autotune(h, not args.no_autotune)   # the launch settings of the timed estimates
        # first use: workspace allocation and tuning.  Every step's seed is estimated once beforehand, so that
        # the autotuner's trials for the launch shapes its sample counts give lie outside the timed region.
        for s in range(args.steps):
            M.mlmc_set_seed(h, 2000 + s)
            M.mlmc_estimate(h, opts())
        for s in range(args.steps):
            M.mlmc_profile_reset(h)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            M.mlmc_set_seed(h, 2000 + s)
            res = M.mlmc_estimate(h, opts())
            float(res.estimate)
            torch.cuda.synchronize()
            e2e_s.append(time.perf_counter() - t0)
            p = M.mlmc_profile_get(h)
            h2d, d2h = p["h2d_bytes"], p["d2h_bytes"]
    finally:
        M.mlmc_destroy(h)

    # the other configurations (one GPU only: the scaling runs time the headline workload alone)
    extras = {}
    if world == 1 and not args.no_extras and args.case == "mlmc":
        with ClockSampler(local) as clk_x:
            m7, r7, _, p7 = timed_runs(WORKLOAD7, TOL7, M.MLMC_FORM_MIXED, args.steps, args.warmup, SEED, True)
            f7 = {} if args.no_fp64 else fp64_forms(WORKLOAD7, TOL7)
            t7 = sum(m7) / len(m7) / 1e3
            extras["cfg5_7level"] = {
                "workload": DESC7, "seconds": t7, "steps": len(m7), "rmse": r7[-1]["rmse"], "N_l": r7[-1]["N"],
                "delta_l": r7[-1]["delta"], "prec_l": r7[-1]["prec"], "fp64_retries_l": r7[-1]["fp64_retries"],
                "solved_dof_per_s": sum(r7[-1]["dofs"]) / t7,
                "solve_gbs": p7["solve_bytes"] / (p7["solve_ms"] * 1e-3) / 1e9 if p7["solve_ms"] > 0 else None,
                "fp64": f7,
                "speedup_vs_fp64_fixed": (f7["fp64_fixed_1e-10"]["seconds"] / t7) if f7 else None,
                "speedup_vs_fp64_adaptive": (f7["fp64_adaptive"]["seconds"] / t7) if f7 else None}
            sw = {}
            for prec in ("FP32", "FP16S", "BF16S", "FP64"):
                sw[prec] = sweep_case(M, torch, dev, args, hbm_peak, peak_src, flush, stream, prec=prec)
            extras["cfg3_sweep"] = sw
            extras["cfg4_adjoint"] = adjoint_case(M, torch, dev, args, hbm_peak, peak_src, flush, stream)
        extras["clocks"] = clk_x.summary()

    line = None
    if rank == 0:
        achieved = prof["solve_bytes"] / (prof["solve_ms"] * 1e-3) / 1e9 if prof["solve_ms"] > 0 else 0.0
        kl_gbs = prof["kl_bytes"] / (prof["kl_ms"] * 1e-3) / 1e9 if prof["kl_ms"] > 0 else 0.0
        kl_tf = prof["kl_flops"] / (prof["kl_ms"] * 1e-3) / 1e12 if prof["kl_ms"] > 0 else 0.0
        step_s = ms_per_step / 1e3
        line = {
            "metric": METRIC, "value": step_s, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            **({"case": "mlmc7"} if args.case == "mlmc7" else {}),
            "config": {"workload": workload_desc(), "l2": "flushed between timed steps (512 MiB write)",
                       "seed": "%d + rank" % SEED, "parallelism": "replicas" if world > 1 else "single GPU"},
            "solved_dof_per_s": dofs / step_s,
            "rmse": [r["rmse"] for r in results], "N_l": results[-1]["N"], "rounds": results[-1]["rounds"],
            "delta_l": results[-1]["delta"], "prec_l": results[-1]["prec"],
            "fp64_retries_l": results[-1]["fp64_retries"],
            "inner_iters_per_step": sum(iters) / len(iters),
            "fp64": fp64,
            "speedup_vs_fp64_fixed": (fp64["fp64_fixed_1e-10"]["seconds"] / step_s) if fp64 else None,
            "speedup_vs_fp64_adaptive": (fp64["fp64_adaptive"]["seconds"] / step_s) if fp64 else None,
            "roofline": {"bound": "hbm", "kernel": "resident_solve", "achieved": achieved, "peak": hbm_peak,
                         "unit": "GB/s", "frac": achieved / hbm_peak, "peak_source": peak_src + " (burst copy)",
                         "traffic": SOLVE_TRAFFIC_BYTES_PER_LAUNCH,
                         "algorithmic_bytes_per_launch": prof["solve_bytes"] / max(1, prof["solve_launches"]),
                         "launches": prof["solve_launches"],
                         "launch_ms_summed_per_step": prof["solve_ms"] / args.steps,
                         "busy_ms_per_step": prof["solve_busy_ms"] / args.steps,
                         "share_of_step": prof["solve_busy_ms"] / sum(ms) if sum(ms) > 0 else None},
            "kl_synthesis": {"achieved_gbs": kl_gbs, "tensor_tflops": kl_tf, "ms_per_step": prof["kl_ms"] / args.steps},
            "autotune": prof["autotune"],
            "e2e": {"value": sum(e2e_s) / len(e2e_s), "unit": "s", "context_create_s": create_s, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            **extras,
        }
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            procs = min(64, os.cpu_count() or 1)
            pool = oracle_pool(procs)
            try:
                oracle_warm(pool, procs, WORKLOAD, SEED)
                secs, ores = oracle_estimate(pool, procs, WORKLOAD, TOL, SEED)
            finally:
                pool.close()
                pool.join()
            line["cpu_baseline"] = {"value": secs, "unit": "s", "cores": procs, "kind": "oracle",
                                    "sample": "one whole estimate: Alg. 4.1 on the same hierarchy and seed "
                                              "(N_l = %s), every fine and coarse solve by FP64 banded Cholesky"
                                              % [int(x) for x in ores["N"]]}
        print(json.dumps(line))
    return 0


def kl_synth_case(M, torch, dev, args, hbm_peak, peak_src, flush, stream):
    """Tensor-core KL synthesis alone: S samples on the 512 x 512 grid, K = 128, corr 0.1, FP32 output
    (--kl-prec FP32) or the FP64 output of the exact-lead form (--kl-prec FP64TC).  Timed twice: into
    rows padded to whole 128-byte lines (the layout the estimate uses; the main numbers) and into the
    dense [S][(n+1)^2] layout ("dense")."""
    S, n, K = args.kl_samples, 512, 128
    V = (n + 1) ** 2
    fprec = getattr(M, "MLMC_" + args.kl_prec)
    prob = M.make_problem(n0=n, m=2, L_max=0, kind=0, K=K, sigma2=1.0, corr_len=0.1, seed=7)
    dt = torch.float32 if fprec == M.MLMC_FP32 else torch.float64

    def run(ld):
        h = M.mlmc_create(prob, dev.index or 0)
        try:
            M.mlmc_profile_enable(h, True)
            a = torch.empty((S, ld), dtype=dt, device=dev)
            xi = torch.empty((S, K), dtype=torch.float64, device=dev)
            M.mlmc_sample_fields(h, 0, 0, S, xi, a, fprec, a_ld=ld)
            for s in range(args.warmup + args.steps):
                if s == args.warmup:
                    M.mlmc_profile_reset(h)
                flush.fill_(float(s))
                M.mlmc_synthesize_fields(h, 0, S, xi, a, fprec, a_ld=ld)
            prof = M.mlmc_profile_get(h)
        finally:
            M.mlmc_destroy(h)
        ms = prof["kl_ms"] / prof["kl_launches"]
        gbs = prof["kl_bytes"] / prof["kl_launches"] / (ms * 1e-3) / 1e9
        tf = prof["kl_flops"] / prof["kl_launches"] / (ms * 1e-3) / 1e12
        return {"row_pitch": ld, "ms_per_launch": ms, "algorithmic_bytes_per_launch": prof["kl_bytes"] / prof["kl_launches"],
                "achieved_gbs": gbs, "hbm_frac": gbs / hbm_peak, "executed_tensor_tflops": tf}

    al = max(32, args.kl_pitch_align)
    padded = run(args.kl_pitch if args.kl_pitch >= V else (V + al - 1) // al * al)
    dense = run(V)
    print(json.dumps(dict({"case": "kl-synth", "prec": args.kl_prec, "samples": S, "n": n, "K": K,
                           "layout": "rows padded to whole 128-byte lines"}, **padded,
                          dense=dense, peak_source=peak_src)))
    return 0


def solve_l4_case(M, torch, dev, args, prob, hbm_peak, peak_src, flush, stream):
    """The dominant launch of the workload in isolation: the finest level's 100 fine systems
    (n = 256) with the accuracy and inner precision the rule assigns to level 4."""
    S, level, n = N_INIT, WORKLOAD["L_max"], WORKLOAD["n0"] * WORKLOAD["m"] ** WORKLOAD["L_max"]
    hs = [1.0 / (WORKLOAD["n0"] * WORKLOAD["m"] ** l) for l in range(level + 1)]
    deltas, precs = M.mlmc_adapt_precision(hs, 0.05)
    h = M.mlmc_create(prob, dev.index or 0)
    try:
        M.mlmc_profile_enable(h, True)
        M.mlmc_debug_set_solve_ring(h, args.ring)
        M.mlmc_set_precond(h, M.MLMC_PC_MG if args.pc == "mg" else M.MLMC_PC_JACOBI, args.mg_nu, args.mg_coarse)
        if args.mg_min:
            M.mlmc_set_mg_coarsest(h, args.mg_min)
        M.mlmc_set_inner_tolerance(h, 0.0, args.tau_min)
        a = torch.empty((S, (n + 1) ** 2), dtype=torch.float32, device=dev)
        Q = torch.empty(S, dtype=torch.float64, device=dev)
        it = torch.empty(S, dtype=torch.int32, device=dev)
        ms = []
        for s in range(args.warmup + args.steps):
            if s == args.warmup:
                M.mlmc_profile_reset(h)
            flush.fill_(float(s))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            M.mlmc_sample_fields(h, level, s * S, S, None, a, M.MLMC_FP32)
            M.mlmc_level_solve(h, n, S, a, M.MLMC_FP32, n, precs[level], M.MLMC_CG, deltas[level], 200000,
                               None, Q, it)
            e1.record(stream)
            e1.synchronize()
            if s >= args.warmup:
                ms.append(e0.elapsed_time(e1))
        prof = M.mlmc_profile_get(h)
    finally:
        M.mlmc_destroy(h)
    achieved = prof["solve_bytes"] / (prof["solve_ms"] * 1e-3) / 1e9
    print(json.dumps({"case": "solve-l4", "ring": args.ring, "mg_min": args.mg_min, "pc": args.pc, "mg_nu": args.mg_nu, "tau_min": args.tau_min,
                      "mg_coarse": args.mg_coarse, "ms_per_step": sum(ms) / len(ms), "systems": S, "n": n,
                      "delta": deltas[level], "prec": precs[level],
                      "inner_iters_per_system": prof["inner_iters"] / (S * args.steps),
                      "solve_ms_per_launch": prof["solve_ms"] / prof["solve_launches"],
                      "algorithmic_bytes_per_launch": prof["solve_bytes"] / prof["solve_launches"],
                      "achieved_gbs": achieved, "peak_gbs": hbm_peak, "frac": achieved / hbm_peak,
                      "peak_source": peak_src}))
    return 0


def fixed3_case(M, torch, dev, args, flush, stream):
    """Fixed-sample FP64 MLMC on 3 levels (h = 1/8, 1/16, 1/32), K = 16, sigma^2 = 1, corr 0.3,
    N_l = 1000 / 500 / 250 solved to a relative residual of 1e-10: the small parity configuration,
    timed."""
    import ctypes
    prob = M.make_problem(n0=8, m=2, L_max=2, kind=0, K=16, sigma2=1.0, corr_len=0.3, seed=0)
    N = (ctypes.c_int64 * 3)(1000, 500, 250)
    h = M.mlmc_create(prob, dev.index or 0)
    try:
        o = M.mlmc_default_options()
        o.form, o.fixed_delta, o.L_start = M.MLMC_FORM_FP64_FIXED, 1e-10, 2
        o.fixed_N = ctypes.cast(N, ctypes.POINTER(ctypes.c_int64))
        ms = []
        for s in range(args.warmup + args.steps):
            flush.fill_(float(s))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = M.result_dict(M.mlmc_estimate(h, o))
            e1.record(stream)
            e1.synchronize()
            if s >= args.warmup:
                ms.append(e0.elapsed_time(e1))
    finally:
        M.mlmc_destroy(h)
    print(json.dumps({"case": "fixed3", "seconds": sum(ms) / len(ms) / 1e3, "N_l": r["N"],
                      "estimate": r["estimate"], "rmse": r["rmse"], "inner_iters": r["inner_iters"]}))
    return 0


def paper_case(M, torch, dev, args, flush, stream):
    """The paper's own MINRES experiment (Sec. 5.1): f = 1, the field of Eq. (5.2) with s = 4 terms,
    q = 2, sigma = 2, h_0 = 1/8, m = 2, Q = int u, Alg. 4.1 with adaptive L (at most 6 levels), k_p = 0.05,
    TOL^2 = 8, 4, 2, 1 x 1e-6.  As in the paper, both estimators solve with FP64 MINRES stopped on the
    relative residual (Jacobi-preconditioned here; the paper's preconditioner is unstated): MPML with the
    adaptive delta_l of Eq. (4.12), standard MLMC with the fixed tolerance 1e-6 (and 1e-10).  Cost is
    the library's count of the solves' arithmetic operations, averaged over --paper-runs seeds; the
    paper reports a FLOP gain of about 1.5 (Sec. 5.1).  The GPU-native form (FP32 inner arithmetic,
    V-cycle preconditioned CG) is timed beside them."""
    import math
    prob_kw = dict(n0=8, m=2, L_max=5, kind=1, K=4, sigma2=4.0, q=2.0, corr_len=0.3)
    forms = [("mpml_fp64_minres", M.MLMC_FORM_FP64_ADAPTIVE, 0.0, M.MLMC_MINRES, M.MLMC_PC_JACOBI),
             ("mlmc_fp64_minres_1e-6", M.MLMC_FORM_FP64_FIXED, 1e-6, M.MLMC_MINRES, M.MLMC_PC_JACOBI),
             ("mlmc_fp64_minres_1e-10", M.MLMC_FORM_FP64_FIXED, 1e-10, M.MLMC_MINRES, M.MLMC_PC_JACOBI),
             ("mpml_gb300_mixed", M.MLMC_FORM_MIXED, 0.0, M.MLMC_CG, M.MLMC_PC_MG)]
    out = {"case": "paper", "runs": args.paper_runs,
           "setting": "Sec. 5.1: Eq. (5.2) field s=4, q=2, sigma=2; h0=1/8, m=2; k_p=0.05; adaptive L <= 5",
           "paper_flop_gain": 1.5, "results": {}}
    for tol2 in (8e-6, 4e-6, 2e-6, 1e-6):
        tol = math.sqrt(tol2)
        per = {}
        for name, form, fd, solver, pc in forms:
            fl, sec, est, Ls, Ns = [], [], [], [], []
            for run in range(args.paper_runs):
                h = M.mlmc_create(M.make_problem(seed=2025 + run, **prob_kw), dev.index or 0)
                try:
                    M.mlmc_set_precond(h, pc)
                    o = M.mlmc_default_options()
                    o.tol, o.form, o.solver = tol, form, solver
                    if fd > 0:
                        o.fixed_delta = fd
                    M.mlmc_estimate(h, o)                     # warm-up (allocations)
                    M.mlmc_profile_enable(h, True)
                    M.mlmc_profile_reset(h)
                    flush.fill_(float(run))
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    r = M.result_dict(M.mlmc_estimate(h, o))
                    e1.record(stream)
                    e1.synchronize()
                    prof = M.mlmc_profile_get(h)
                finally:
                    M.mlmc_destroy(h)
                fl.append(prof["solve_flops"])
                sec.append(e0.elapsed_time(e1) / 1e3)
                est.append(r["estimate"])
                Ls.append(r["L"])
                Ns.append(r["N"])
            per[name] = {"flops": sum(fl) / len(fl), "seconds": sum(sec) / len(sec),
                         "estimate": sum(est) / len(est), "L_mean": sum(Ls) / len(Ls),
                         "N_l_first_run": Ns[0]}
        base = per["mlmc_fp64_minres_1e-6"]
        for name in per:
            per[name]["flop_gain_vs_mlmc_1e-6"] = base["flops"] / per[name]["flops"]
            per[name]["time_gain_vs_mlmc_1e-6"] = base["seconds"] / per[name]["seconds"]
        out["results"]["TOL2=%g" % tol2] = per
    out["cholesky"] = paper_cholesky(M, torch, dev, args, flush, stream, prob_kw)
    return out


def paper_cholesky(M, torch, dev, args, flush, stream, prob_kw):
    """The paper's direct-solver experiment (Sec. 5.2): the same field and hierarchy, MPML solving with a
    banded Cholesky factor in low precision and iterative refinement (Table 1, right: hhss on level 0,
    ssss on level 1, ssdd above) against standard MLMC with an FP64 factor (dddd), both on the sample
    counts of an adaptive standard-MLMC run and the same seeds.  Cost: the memory model of Sec. 5.2
    (bits of every factor and vector entry computed and stored; the paper reports about 2x) beside the
    measured time."""
    import ctypes
    import math
    out = {"paper_memory_gain": 2.0, "results": {}}
    for tol2 in (8e-6, 4e-6, 2e-6, 1e-6):
        tol = math.sqrt(tol2)
        bits = {"mpml": [], "mlmc": []}
        secs = {"mpml": [], "mlmc": []}
        for run in range(args.paper_runs):
            kw = dict(prob_kw, L_max=3, seed=2025 + run)
            h = M.mlmc_create(M.make_problem(**kw), dev.index or 0)
            try:
                o = M.mlmc_default_options()
                o.tol, o.form, o.solver, o.fixed_delta = tol, M.MLMC_FORM_FP64_FIXED, M.MLMC_CHOLESKY, 1e-10
                r0 = M.result_dict(M.mlmc_estimate(h, o))        # sample counts of the adaptive MLMC run
            finally:
                M.mlmc_destroy(h)
            Nl = [int(x) for x in r0["N"][: r0["L"] + 1]]
            arr = (ctypes.c_int64 * len(Nl))(*Nl)
            for name, form in (("mpml", M.MLMC_FORM_MIXED), ("mlmc", M.MLMC_FORM_FP64_FIXED)):
                h = M.mlmc_create(M.make_problem(**kw), dev.index or 0)
                try:
                    o = M.mlmc_default_options()
                    o.form, o.solver, o.fixed_delta, o.L_start = form, M.MLMC_CHOLESKY, 1e-10, len(Nl) - 1
                    o.fixed_N = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int64))
                    M.mlmc_estimate(h, o)
                    M.mlmc_profile_enable(h, True)
                    M.mlmc_profile_reset(h)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    M.mlmc_estimate(h, o)
                    e1.record(stream)
                    e1.synchronize()
                    prof = M.mlmc_profile_get(h)
                finally:
                    M.mlmc_destroy(h)
                bits[name].append(prof["chol_bits"])
                secs[name].append(e0.elapsed_time(e1) / 1e3)
        out["results"]["TOL2=%g" % tol2] = {
            "memory_gain": sum(bits["mlmc"]) / sum(bits["mpml"]),
            "time_gain": sum(secs["mlmc"]) / sum(secs["mpml"]),
            "mpml_seconds": sum(secs["mpml"]) / len(secs["mpml"]),
            "mlmc_seconds": sum(secs["mlmc"]) / len(secs["mlmc"])}
    out["quarter"] = paper_cholesky_quarter(M, torch, dev, args, stream)
    return out


def paper_cholesky_quarter(M, torch, dev, args, stream):
    """The quarter-precision variant of Sec. 5.2: s = 1 term, sigma = 1, q = 2, h_0 = 1/4, levels 0 to 3,
    k_p = 0.4, MSE tolerance 2e-6; MPML solves with qhhh on level 0 (an FP8 E4M3 factor, the q43 format)
    and hhss above, against an FP64 factor (dddd) on the sample counts of an adaptive standard-MLMC run and
    the same seeds.  The paper reports a memory gain of about 3.5 and an MPML error 11 % above MLMC's."""
    import ctypes
    import math
    kw = dict(n0=4, m=2, L_max=3, kind=1, K=1, sigma2=1.0, q=2.0, corr_len=0.3)
    tol = math.sqrt(2e-6)
    bits = {"mpml": [], "mlmc": []}
    secs = {"mpml": [], "mlmc": []}
    est = {"mpml": [], "mlmc": []}
    flags = 0
    for run in range(args.paper_runs):
        kwr = dict(kw, seed=3025 + run)
        h = M.mlmc_create(M.make_problem(**kwr), dev.index or 0)
        try:
            o = M.mlmc_default_options()
            o.tol, o.form, o.solver, o.fixed_delta = tol, M.MLMC_FORM_FP64_FIXED, M.MLMC_CHOLESKY, 1e-10
            o.kp = 0.4
            r0 = M.result_dict(M.mlmc_estimate(h, o))
        finally:
            M.mlmc_destroy(h)
        Nl = [int(x) for x in r0["N"][: r0["L"] + 1]]
        arr = (ctypes.c_int64 * len(Nl))(*Nl)
        for name, form in (("mpml", M.MLMC_FORM_MIXED), ("mlmc", M.MLMC_FORM_FP64_FIXED)):
            h = M.mlmc_create(M.make_problem(**kwr), dev.index or 0)
            try:
                o = M.mlmc_default_options()
                o.form, o.solver, o.fixed_delta, o.L_start = form, M.MLMC_CHOLESKY, 1e-10, len(Nl) - 1
                o.kp, o.tol, o.chol_table = 0.4, tol, 1
                o.fixed_N = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int64))
                M.mlmc_estimate(h, o)
                M.mlmc_profile_enable(h, True)
                M.mlmc_profile_reset(h)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = M.result_dict(M.mlmc_estimate(h, o))
                e1.record(stream)
                e1.synchronize()
                prof = M.mlmc_profile_get(h)
            finally:
                M.mlmc_destroy(h)
            bits[name].append(prof["chol_bits"])
            secs[name].append(e0.elapsed_time(e1) / 1e3)
            est[name].append(r["estimate"])
            flags |= r["flags_or"]
    diff = [abs(a - b) for a, b in zip(est["mpml"], est["mlmc"])]
    return {"setting": "Sec. 5.2 quarter precision: s=1, sigma=1, q=2, h0=1/4, levels 0-3, k_p=0.4, TOL^2=2e-6; "
                       "qhhh on level 0 (FP8 E4M3 factor), hhss above",
            "paper_memory_gain": 3.5, "memory_gain": sum(bits["mlmc"]) / sum(bits["mpml"]),
            "time_gain": sum(secs["mlmc"]) / sum(secs["mpml"]),
            "mean_abs_estimate_diff": sum(diff) / len(diff), "flags_or": flags}


def adjoint_case(M, torch, dev, args, hbm_peak, peak_src, flush, stream):
    """Adjoint gradients dQ/dxi: 1024 samples on the 256 x 256 grid, K = 256, corr 0.1, QoI the
    integral over [0.25, 0.75]^2; forward and adjoint solves (FP32 inner, FP64 refinement to
    1e-8) in one launch, then the element products and the contraction onto the KL terms."""
    S, n, K = 1024, 256, 256
    prob = M.make_problem(n0=n, m=2, L_max=0, kind=0, K=K, sigma2=1.0, corr_len=0.1, seed=21, qoi=1,
                          box=(0.25, 0.75, 0.25, 0.75))
    h = M.mlmc_create(prob, dev.index or 0)
    try:
        M.mlmc_profile_enable(h, True)
        M.mlmc_set_autotune(h, not args.no_autotune)
        xi = torch.empty((S, K), dtype=torch.float64, device=dev)
        a = torch.empty((S, (n + 1) ** 2), dtype=torch.float32, device=dev)
        M.mlmc_sample_fields(h, 0, 0, S, xi, a, M.MLMC_FP32)
        Q = torch.empty(S, dtype=torch.float64, device=dev)
        G = torch.empty((S, K), dtype=torch.float64, device=dev)
        ms = []
        for s in range(args.warmup + args.steps):
            if s == args.warmup:
                M.mlmc_profile_reset(h)
            flush.fill_(float(s))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            M.mlmc_adjoint_grad(h, 0, S, xi, M.MLMC_FP32, 1e-8, 200000, Q, G)
            e1.record(stream)
            e1.synchronize()
            if s >= args.warmup:
                ms.append(e0.elapsed_time(e1))
        prof = M.mlmc_profile_get(h)
    finally:
        M.mlmc_destroy(h)
    t = sum(ms) / len(ms) / 1e3
    achieved = prof["solve_bytes"] / (prof["solve_ms"] * 1e-3) / 1e9 if prof["solve_ms"] > 0 else 0.0
    return {"case": "adjoint", "samples": S, "n": n, "K": K, "seconds_per_batch": t, "steps": len(ms),
            "grads_per_s": S / t, "solve_share": prof["solve_busy_ms"] / (sum(ms)),
            "solve_achieved_gbs": achieved, "peak_gbs": hbm_peak, "solve_frac": achieved / hbm_peak,
            "peak_source": peak_src}


def sweep_case(M, torch, dev, args, hbm_peak, peak_src, flush, stream, prec=None):
    """Single-level batched solve: S systems on the 512 x 512 grid (261,121 unknowns each), KL field
    with K = 128 terms and correlation length 0.1, fixed relative residual 1e-6; solved DOF/s and
    the solve kernel's HBM rate."""
    S, n, K, delta = args.sweep_samples, 512, 128, args.sweep_delta
    pname = prec or args.prec
    prec = getattr(M, "MLMC_" + pname)
    fp64 = prec == M.MLMC_FP64
    prob = M.make_problem(n0=n, m=2, L_max=0, kind=0, K=K, sigma2=1.0, corr_len=0.1, seed=11)
    h = M.mlmc_create(prob, dev.index or 0)
    try:
        M.mlmc_profile_enable(h, True)
        M.mlmc_debug_set_solve_ring(h, args.ring)
        M.mlmc_set_precond(h, M.MLMC_PC_MG if args.pc == "mg" else M.MLMC_PC_JACOBI, args.mg_nu, args.mg_coarse)
        M.mlmc_set_autotune(h, not args.no_autotune)
        a = torch.empty((S, (n + 1) ** 2), dtype=torch.float64 if fp64 else torch.float32, device=dev)
        Q = torch.empty(S, dtype=torch.float64, device=dev)
        it = torch.empty(S, dtype=torch.int32, device=dev)
        fl = torch.empty(S, dtype=torch.int32, device=dev)
        fprec = M.MLMC_FP64 if fp64 else M.MLMC_FP32
        M.mlmc_sample_fields(h, 0, 0, S, None, a, fprec)
        ms = []
        for s in range(args.warmup + args.steps):
            if s == args.warmup:
                M.mlmc_profile_reset(h)
            flush.fill_(float(s))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            M.mlmc_level_solve(h, n, S, a, fprec, n, prec, M.MLMC_CG, delta, 200000, None, Q, it, None, fl)
            e1.record(stream)
            e1.synchronize()
            if s >= args.warmup:
                ms.append(e0.elapsed_time(e1))
        prof = M.mlmc_profile_get(h)
        flags = fl.cpu()
    finally:
        M.mlmc_destroy(h)
        del a
        torch.cuda.empty_cache()
    t = sum(ms) / len(ms) / 1e3
    achieved = prof["solve_bytes"] / (prof["solve_ms"] * 1e-3) / 1e9
    return {"case": "sweep", "prec": pname, "ring": args.ring, "systems": S, "n": n, "delta": delta,
            "seconds_per_batch": t, "steps": len(ms), "solved_dof_per_s": S * (n - 1) ** 2 / t,
            "inner_iters_per_system": prof["inner_iters"] / (S * args.steps),
            "algorithmic_bytes_per_launch": prof["solve_bytes"] / prof["solve_launches"],
            "achieved_gbs": achieved, "peak_gbs": hbm_peak, "frac": achieved / hbm_peak,
            "peak_source": peak_src, "all_converged": bool((flags == M.MLMC_F_CONVERGED).all())}


if __name__ == "__main__":
    sys.exit(main())
