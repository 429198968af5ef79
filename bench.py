#!/usr/bin/env python3
"""Benchmark of the multilevel spectral DD hot path on one GB300.

A step is one pass of the whole hot path on the 2D 512 x 512 Q1 workload
(GRF background x channels/inclusions, contrast 1e6, 16 x 16 subdomains,
overlap 2, three levels, nev <= 12, eta = 0.3): hierarchy set-up (fine
Dirichlet factorisations, shifted-Neumann factorisations, batched subspace
iterations, coarse Galerkin and generating-system GEVPs, coarsest factor)
followed by PCG to relative residual 1e-8.  The metric is seconds per step of
the chosen form (FP32 fine factors and solves, FP64 elsewhere); the plain FP64
form is timed beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).
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

METRIC = "setup+PCG seconds to rel. residual 1e-8, chosen vs plain FP64 form; % roofline"
TOL = 1e-8
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
FP64_PEAK_TFLOPS_NOMINAL = 1.25     # GB300 FP64, nominal (used only for "alu"-bound kernels)


def measured_traffic(family, workload_name):
    """DRAM traffic of the family's kernel from the committed ncu summary
    (profiles/traffic.txt: key=value lines).  The figure holds only for the
    workload and the kernel source it was captured from: absent for another
    workload, null when the source file's SHA-256 differs."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        kv = dict(line.strip().split("=", 1) for line in open(path) if "=" in line and not line.startswith("#"))
    except OSError:
        return {}
    if kv.get("family") != family or kv.get("workload") != workload_name:
        return {}
    src = os.path.join(ROOT, kv.get("source", ""))
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return {}
    if digest != kv.get("source_sha256"):
        return {"traffic": None, "traffic_note": "kernel source changed since the ncu capture"}
    return {"traffic": float(kv["dram_bytes_per_launch"]),
            "traffic_launch_algorithmic_bytes": float(kv["algorithmic_bytes_captured_launch"]),
            "traffic_kernel": kv.get("kernel"), "traffic_source": "profiles/traffic.txt"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["grf512", "channels64", "composite128", "composite96", "batch256"],
                    default="grf512")
    ap.add_argument("--batch-count", type=int, default=256, help="batch256: number of problems")
    ap.add_argument("--oracle-sample", type=int, default=16,
                    help="3D workload: fine subdomains in the CPU oracle's bounded sample")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the CPU oracle step (and the error summary against it)")
    ap.add_argument("--oracle-leg", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--forms", choices=["both", "chosen"], default="both",
                    help="chosen: time only the chosen form (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-solvers", action="store_true",
                    help="skip the PCG / hybrid-GMRES comparison after the timed steps")
    ap.add_argument("--no-breakdown", action="store_true",
                    help="skip the extra all-families profiled step (profiling runs: one step only)")
    return ap.parse_args()


def max_over_ranks(value, dist=None, device=None):
    """The job's time is that of its slowest rank: the largest value over all
    ranks of the process group (a CPU tensor for gloo, a device tensor for
    NCCL); the value itself with no process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def solver_leg(H, b, steps, warmup, sync):
    """Median wall time per solve (ms, synchronised on both sides) of PCG with
    the additive preconditioner and of flexible GMRES with the hybrid one on
    the same hierarchy, with iterations and residuals.  Outside the timed
    step; a failure is recorded, not raised."""
    out = {}
    for name, f in (("pcg_additive", lambda: H.solve(b, tol=TOL, allow_maxit=True)),
                    ("gmres_hybrid", lambda: H.solve_gmres(b, tol=TOL, allow_maxit=True))):
        try:
            for _ in range(warmup):
                f()
            ts, it, rel = [], 0, float("nan")
            for _ in range(max(1, steps)):
                sync()
                t0 = time.perf_counter()
                _, it, rel = f()
                sync()
                ts.append(time.perf_counter() - t0)
            out[name] = {"ms": round(1e3 * statistics.median(ts), 3), "iterations": int(it),
                         "rel_residual": float(rel)}
        except Exception as e:                                    # recorded in the JSON line
            out[name] = {"error": repr(e)[:200]}
    out["note"] = ("one hierarchy of the chosen form; pcg rel_residual is the recursive residual, "
                   "gmres rel_residual the true residual (FP64 attainable accuracy ~1e-6 here)")
    return out


def workload(name, seed):
    import synthetic_inputs as si
    return {"grf512": si.grf512, "channels64": si.channels64, "composite128": si.composite128,
            "composite96": si.composite96}[name](seed=seed)


def full_oracle_step(wname):
    """The 3D composite workload is too large for a full oracle step on the
    host (512 band factorisations of order 6859, half-bandwidth 381, with
    their subspace iterations: minutes on 16 cores); it gets a bounded
    sample instead."""
    return wname not in ("composite128", "composite96")


# ------------------------------------------------------------------ CPU oracle step
def workload_config(w, unknowns, world):
    """The config object of the JSON line (the same for both arms)."""
    return {"workload": w.name, "n_elements": list(w.n), "unknowns": int(unknowns), "subdomains": list(w.parts),
            "overlap": w.overlap, "levels": w.levels, "nev_max": w.nev_max, "eta": w.eta, "tol": TOL,
            "form": "chosen (precision=1)", "l2": "flushed between steps (512 MB write)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def save_gpu_results(pkg, w, kappa, b):
    """Selected Ritz values and counts of every fine and middle subdomain,
    level dimensions, and the PCG solution of one chosen-form hierarchy
    (bench defaults), written to a temporary .npz for the oracle leg."""
    import numpy as np
    H = pkg.Hierarchy(w.n, kappa, w.parts, w.overlap, w.levels, w.group, w.nev_max, w.eta,
                      dirichlet_faces=w.dirichlet_faces, precision=1)
    x, it, _ = H.solve(b, tol=TOL)
    st = H.stats()
    out = {"level_dim": np.array(st["level_dim"]), "iterations": np.array(it), "x": x.cpu().numpy()}
    L = w.levels - 1
    for name, lev in (("fine", L), ("middle", 1)):
        if name == "middle" and L < 2:
            continue
        P = st["subdomains"][lev]
        lam = np.full((P, 32), np.nan)
        ms = np.zeros(P, dtype=np.int64)
        for i in range(P):
            th, m = H.eigenvalues(lev, i)
            lam[i, :len(th)] = th
            ms[i] = m
        out["%s_lam" % name], out["%s_m" % name] = lam, ms
    H.close()
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    np.savez(path, **out)
    return path


def oracle_step(wname, processes):
    """One full step of the CPU oracle in method mode on the workload: set-up
    (assembly, decomposition, band Cholesky factors and block subspace
    iteration on every fine subdomain in `processes` spawned worker
    processes, dense generating-system GEVPs on the middle level, Galerkin
    and coarsest factors) and PCG with the additive preconditioner to
    relative residual 1e-8.  Returns (seconds, result dict)."""
    from oracle import fem, method, method_mode
    w = workload(wname, 0)
    t0 = time.perf_counter()
    mesh = fem.Mesh(w.n, w.dirichlet_faces)
    kap = w.coefficient()
    H = method_mode.MethodModeHierarchy(mesh, kap, w.parts, w.overlap, w.levels, w.group, w.nev_max, w.eta,
                                        processes=processes)
    t1 = time.perf_counter()
    b = fem.load_vector(mesh)
    x, it, *_ = method.pcg(H.A, b, H.apply_preconditioner, TOL)
    t2 = time.perf_counter()
    return t2 - t0, dict(H=H, x=x, b=b, iterations=it, setup_s=t1 - t0, pcg_s=t2 - t1)


def error_vs_oracle(gpu, res, eta):
    """Errors of the GPU's chosen form against the oracle's method-mode
    results on the same workload: selected eigenvalues (relative, floor
    1e-3 eta) and counts on the fine and middle levels, coarse dimensions,
    CG iterations, and both solutions against a sparse direct solve."""
    import numpy as np
    import scipy.sparse.linalg as spla
    H = res["H"]
    out = {}
    for name, lev in (("fine", H.L), ("middle", 1)):
        if lev < 1 or lev > H.L or (name == "middle" and H.L < 2):
            continue
        subs = H.levels[lev].subs
        g_l, g_m = gpu["%s_lam" % name], gpu["%s_m" % name]
        worst, mism = 0.0, []
        for i, s in enumerate(subs):
            if int(g_m[i]) != s["m"]:
                mism.append([i, int(g_m[i]), int(s["m"])])
                continue
            m = s["m"]
            if m:
                lam = np.asarray(s["lam"][:m])
                e = np.abs(g_l[i][:m] - lam) / np.maximum(np.abs(lam), 1e-3 * eta)
                worst = max(worst, float(e.max()))
        out[name] = {"subdomains": len(subs), "max_rel_eig_err": worst, "count_mismatch": mism}
    out["coarse_dims"] = {"gpu": [int(v) for v in gpu["level_dim"]],
                          "oracle": [int(H.coarse_dims()[l]) for l in range(H.L)] + [int(H.n)]}
    out["iterations"] = {"gpu": int(gpu["iterations"]), "oracle": int(res["iterations"])}
    A = H.A.tocsc()
    xd = spla.spsolve(A, res["b"])
    an = lambda v: float(np.sqrt(max(v @ (A @ v), 0.0)))
    for key, x in (("gpu", gpu["x"]), ("oracle", res["x"])):
        out["solution_%s" % key] = {"rel_err_2": float(np.linalg.norm(x - xd) / np.linalg.norm(xd)),
                                    "rel_err_A": an(x - xd) / an(xd)}
    out["note"] = ("oracle = method mode (FP64 band Cholesky + block subspace iteration to eigen-residual 1e-8, "
                   "exact dense GEVPs on the middle level); both CG runs stop at rel. residual 1e-8, so the "
                   "solution errors are those of that stopping rule")
    return out


def oracle_leg(args):
    """Run by bench.py itself in a fresh interpreter after the GPU work: one
    timed oracle step on all host cores, and (given the GPU's results) the
    error summary.  Prints one JSON object."""
    import numpy as np
    procs = os.cpu_count() or 1
    if not full_oracle_step(args.workload):
        secs, res = oracle_fine_sample(args.workload, procs, args.oracle_sample)
        out = {"seconds": secs, "cores": procs, "sample_subdomains": res["sample"], "total_subdomains": res["total"]}
        if args.oracle_leg and os.path.exists(args.oracle_leg):
            g = np.load(args.oracle_leg, allow_pickle=True)
            w = workload(args.workload, 0)
            worst, mism = 0.0, []
            for i, s in zip(res["sample"], res["subs"]):
                m = int(g["fine_m"][i])
                if m != s["m"]:
                    mism.append([int(i), m, int(s["m"])])
                elif m:
                    lam = s["lam"][:m]
                    worst = max(worst, float(np.max(np.abs(g["fine_lam"][i][:m] - lam) / np.maximum(np.abs(lam),
                                                                                              1e-3 * w.eta))))
            out["error_vs_oracle"] = {"fine_sampled": {"subdomains": len(res["sample"]), "max_rel_eig_err": worst,
                                                       "count_mismatch": mism},
                                      "note": "oracle = method mode on the sampled fine subdomains (FP64 band "
                                              "Cholesky + block subspace iteration to eigen-residual 1e-8)"}
        print(json.dumps(out), flush=True)
        return
    secs, res = oracle_step(args.workload, procs)
    out = {"seconds": secs, "setup_s": res["setup_s"], "pcg_s": res["pcg_s"], "iterations": res["iterations"],
           "cores": procs}
    if args.oracle_leg and os.path.exists(args.oracle_leg):
        g = np.load(args.oracle_leg, allow_pickle=True)
        gpu = {k: g[k] for k in g.files}
        w = workload(args.workload, 0)
        try:
            out["error_vs_oracle"] = error_vs_oracle(gpu, res, w.eta)
        except Exception as e:                                    # recorded in the JSON line
            out["error_vs_oracle"] = {"error": repr(e)[:300]}
    print(json.dumps(out), flush=True)


def oracle_fine_sample(wname, processes, count):
    """The oracle's fine-level local set-up (Neumann assembly, partition of
    unity, band Cholesky of Abar_i + sigma B_i, block subspace iteration,
    selection) on `count` fine subdomains spread over the workload, in
    `processes` spawned workers.  Returns (seconds, result dict)."""
    import numpy as np
    from oracle import method_mode
    w = workload(wname, 0)
    P = int(np.prod(w.parts))
    sample = sorted({int(v) for v in np.linspace(0, P - 1, min(count, P))})
    t0 = time.perf_counter()
    subs = method_mode.fine_level_sample(w.n, w.dirichlet_faces, w.coefficient(), w.parts, w.overlap, w.levels,
                                         w.group, w.nev_max, w.eta, sample, processes)
    return time.perf_counter() - t0, {"sample": sample, "total": P, "subs": subs}


def cpu_baseline_obj(res, wname):
    if res is None or "error" in res:
        return {"value": None, "unit": "s", "cores": None, "kind": "oracle",
                "sample": "failed: %s" % (res or {}).get("error", "not run")}
    if "sample_subdomains" in res:
        return {"value": round(res["seconds"], 3), "unit": "s", "cores": res["cores"], "kind": "oracle",
                "sample": ("%s: bounded sample, the oracle's fine-level local set-up (method mode: Neumann "
                           "assembly, band Cholesky, block subspace iteration, selection) of %d of %d fine "
                           "subdomains on %d host cores, after the GPU timed region; the value is that sample's "
                           "time, not a full step") % (wname, len(res["sample_subdomains"]),
                                                       res["total_subdomains"], res["cores"])}
    return {
        "value": round(res["seconds"], 3), "unit": "s", "cores": res["cores"], "kind": "oracle",
        "sample": ("%s: one full oracle step, method mode (the whole workload: set-up %.1f s, PCG %.1f s, "
                   "%d iterations), run after the GPU timed region on all %d host cores (fine subdomains in "
                   "worker processes)") % (wname, res["setup_s"], res["pcg_s"], res["iterations"], res["cores"]),
    }


def run_oracle_leg(args, gpu_npz):
    """Start the oracle leg as a fresh interpreter and parse its JSON line."""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-leg", gpu_npz or "-", "--workload", args.workload,
           "--oracle-sample", str(args.oracle_sample)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=1800)
        for line in reversed(r.stdout.strip().splitlines()):
            if line.startswith("{"):
                return json.loads(line)
        return {"error": "no output (rc %d): %s" % (r.returncode, r.stderr[-300:])}
    except Exception as e:
        return {"error": repr(e)[:300]}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for k, nm in enumerate(names):
                    if r[3 + k].strip().lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__
    __graft_entry__.build()
    import paper_2106_06404_gb300 as pkg
    from paper_2106_06404_gb300 import msdd

    w = workload(args.workload, rank)
    kap_np = w.coefficient()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    with torch.cuda.stream(stream):
        kappa = torch.tensor(kap_np, device=dev)                   # resident in HBM before timing
        b = pkg.assemble_rhs(w.n, w.dirichlet_faces)

        def step(precision, profile):
            H = pkg.Hierarchy(w.n, kappa, w.parts, w.overlap, w.levels, w.group, w.nev_max, w.eta,
                              dirichlet_faces=w.dirichlet_faces, precision=precision, profile=profile)
            x, it, rel = H.solve(b, tol=TOL)
            st = H.stats()
            H.close()
            return it, rel, st

        def timed(precision, profile):
            for _ in range(args.warmup):
                step(precision, False)
            times, its, stats = [], [], None
            barrier()
            l0 = msdd.kernel_launches()
            for _ in range(args.steps):
                flush.fill_(1.0)                                   # evict L2 between steps
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                it, rel, st = step(precision, profile)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
                its.append(it)
                stats = st
            launches = msdd.kernel_launches() - l0
            barrier()
            return times, its, stats, launches

        # timed steps profile only the band-solve families (the roofline kernel);
        # the per-family breakdown comes from one extra step after the timed region
        with ClockSampler(local_rank) as clk:
            t_chosen, it_chosen, st_chosen, launches = timed(1, 2)
        st_families = st_chosen if args.no_breakdown else step(1, 1)[2]
        if args.forms == "both":
            t_plain, it_plain, st_plain, _ = timed(0, False)
        else:
            t_plain, it_plain, st_plain = None, None, None

        # end to end through host buffers: kappa and b copied in, x copied out
        kap_pin = torch.tensor(kap_np).pin_memory()
        b_host = b.cpu().numpy()
        e2e_times = []
        for k in range(0 if args.no_e2e else args.warmup + args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            kd = kap_pin.to(dev, non_blocking=True)
            H = pkg.Hierarchy(w.n, kd, w.parts, w.overlap, w.levels, w.group, w.nev_max, w.eta,
                              dirichlet_faces=w.dirichlet_faces, precision=1)
            x_host, it, rel = H.solve_host(b_host, tol=TOL)
            H.close()
            torch.cuda.synchronize(dev)
            if k >= args.warmup:
                e2e_times.append(time.perf_counter() - t0)

        # solver comparison on one hierarchy (not part of the timed step)
        solvers = None
        if not args.no_solvers:
            try:
                H = pkg.Hierarchy(w.n, kappa, w.parts, w.overlap, w.levels, w.group, w.nev_max, w.eta,
                                  dirichlet_faces=w.dirichlet_faces, precision=1)
                solvers = solver_leg(H, b, args.steps, args.warmup, lambda: torch.cuda.synchronize(dev))
                H.close()
            except Exception as e:
                solvers = {"error": repr(e)[:200]}

        # the chosen form's results for the error summary against the CPU oracle
        gpu_npz = None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            try:
                gpu_npz = save_gpu_results(pkg, w, kappa, b)
            except Exception as e:
                gpu_npz = None
                print("gpu results not saved: %r" % (e,), file=sys.stderr)

    total = max_over_ranks(sum(t_chosen), dist, dev)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel family of the chosen form (live CUDA events)
    prof = st_chosen["prof"]
    # the dominant kernel family with algorithmic amounts attached
    fam = max((k for k in prof if prof[k]["bytes"] > 0 or prof[k]["flops"] > 0), key=lambda k: prof[k]["ms"])
    pf = prof[fam]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    intensity = pf["flops"] / max(pf["bytes"], 1.0)
    fp64_bound = fam.startswith("fine_gevp_update") or fam.startswith("fine_gevp_gram") or \
        (fam.endswith("_solve") and st_chosen["precision"] == 0)
    if fp64_bound:
        achieved = pf["flops"] / (pf["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": FP64_PEAK_TFLOPS_NOMINAL,
                "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS_NOMINAL, 4)}
    else:
        achieved = pf["bytes"] / (pf["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4)}
    roof.update({"kernel": fam, "launches": pf["launches"], "avg_launch_ms": round(pf["ms"] / pf["launches"], 4),
                 "algorithmic_bytes_per_launch": pf["bytes"] / pf["launches"],
                 "algorithmic_flops_per_launch": pf["flops"] / pf["launches"],
                 "arith_intensity_flop_per_byte": round(intensity, 3),
                 "peak_source": "MEASURED_PEAKS.json" if "hbm_gbs" in peaks else "fallback",
                 "traffic": None,
                 # pf holds the family times of one step (the last timed step's
                 # hierarchy): that time over the mean step time
                 "share_of_step": round((pf["ms"] / 1e3) / (total / args.steps), 4)})
    roof.update(measured_traffic(fam, w.name))

    # the CPU oracle: one full step on all host cores, after all GPU work
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = run_oracle_leg(args, gpu_npz)
        if gpu_npz:
            os.unlink(gpu_npz)

    n = st_chosen["n"]
    e2e_val = statistics.mean(e2e_times) if e2e_times else None
    line = {
        "metric": METRIC,
        "value": round(total / args.steps, 6),
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(1e3 * total / args.steps, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 outer / f32 fine factors and solves / double-f32 fine Gram, apply, update",
        "data": "synthetic (seeded GRF x channels/inclusions, contrast 1e6)",
        "config": workload_config(w, n, world),
        "iterations": it_chosen[-1],
        "step_seconds": [round(t, 6) for t in t_chosen],
        "setup_ms": round(st_chosen["setup_ms"], 3),
        "solve_ms": round(st_chosen["solve_ms"], 3),
        "phase_ms": [round(v, 3) for v in st_chosen["phase_ms"][:8]],
        "level_dim": st_chosen["level_dim"],
        "eig_iters_max": st_chosen["eig_iters_max"],
        "plain_fp64": None if t_plain is None else {
            "value": round(sum(t_plain) / args.steps, 6), "unit": "s", "iterations": it_plain[-1],
            "setup_ms": round(st_plain["setup_ms"], 3), "solve_ms": round(st_plain["solve_ms"], 3),
            "step_seconds": [round(t, 6) for t in t_plain]},
        "speedup_chosen_vs_plain": None if t_plain is None else round(sum(t_plain) / max(total, 1e-12), 3),
        "kernel_families_ms": {k: round(v["ms"], 3) for k, v in st_families["prof"].items()},
        "kernel_families_note": "one extra step with every family timed (profile level 1), after the timed region; "
                                "the timed steps time only the band-solve families (level 2)",
        "roofline": roof,
        "clocks": clk.summary(),
        "e2e": {"value": round(e2e_val, 6) if e2e_val else None, "unit": "s",
                "h2d_bytes_per_step": int(kap_np.nbytes + n * 8), "d2h_bytes_per_step": int(n * 8)},
        "gpu_launches": int(launches),
        "cpu_baseline": cpu_baseline_obj(cpu, w.name) if cpu is not None else None,
        "error_vs_oracle": (cpu or {}).get("error_vs_oracle"),
        "solvers": solvers,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    """The reference arm: the CPU oracle, as it stands (method mode), on the
    same workload, config and metric; rank 0 only.  Each timed step is one
    full oracle step (set-up + PCG) on all host cores; the warm-up steps run
    the oracle on the small 64 x 64 channel workload."""
    if rank != 0:
        return
    procs = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_step("channels64", procs)
    vals, last = [], None
    for _ in range(args.steps):
        secs, res = oracle_step(args.workload, procs)
        vals.append(secs)
        last = {"seconds": secs, "setup_s": res["setup_s"], "pcg_s": res["pcg_s"], "iterations": res["iterations"],
                "cores": procs}
        n = res["H"].n
    v = statistics.mean(vals)
    w = workload(args.workload, 0)
    cb = cpu_baseline_obj(last, w.name)
    cb["sample"] = cb["sample"].replace("run after the GPU timed region on", "on")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * v, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, n, world),
        "step_seconds": [round(t, 3) for t in vals],
        "cpu_baseline": dict(cb, value=round(v, 3)),
        "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batch of problems
def run_batch(args):
    """The multi-problem workload: the batch256 recipe (256 independent 2D
    problems of uneven size) set up and solved with msdd_batch_run; a step is
    the whole batch.  The worker count is picked by a timing sweep on the
    first 32 problems (the batch's own tuner)."""
    import numpy as np
    import torch
    import synthetic_inputs as si
    import __graft_entry__
    __graft_entry__.build()
    import paper_2106_06404_gb300 as pkg
    ws = si.batch256(count=args.batch_count)
    probs = []
    for w in ws:
        probs.append(dict(n=w.n, kappa=torch.tensor(w.coefficient(), device="cuda"), parts=w.parts,
                          overlap=w.overlap, levels=w.levels, group=w.group, b=pkg.assemble_rhs(w.n)))
    torch.cuda.synchronize()

    def run(sub, precision, nworkers):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = pkg.batch_run(sub, ws[0].nev_max, ws[0].eta, tol=TOL, precision=precision, nworkers=nworkers)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    tune = {}
    for nw in (4, 8, 16, 32):
        run(probs[:32], 1, nw)
        tune[nw] = run(probs[:32], 1, nw)[0]
    best = min(tune, key=tune.get)
    res = {}
    for prec in (1, 0):
        for _ in range(args.warmup):
            run(probs, prec, best)
        times, out = [], None
        for _ in range(args.steps):
            t, out = run(probs, prec, best)
            times.append(t)
        res[prec] = (times, out)
    t1, (xs, it, rel, st, sms, pms) = res[1]
    t0 = res[0][0]
    n_unknowns = int(sum(x.numel() for x in xs))
    line = {
        "metric": METRIC, "value": round(statistics.mean(t1), 6), "unit": "s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(t1), 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 outer / f32 fine factors and solves / double-f32 fine Gram, apply, update",
        "data": "synthetic (batch recipe: seeded sides 128-384, 4x4-12x12 subdomains, log-normal x channels 1e4-1e6)",
        "config": {"workload": "batch2d_%dproblems" % len(ws), "problems": len(ws), "unknowns": n_unknowns,
                   "levels": 2, "nev_max": ws[0].nev_max, "eta": ws[0].eta, "tol": TOL, "form": "chosen (precision=1)",
                   "parallelism": "single GPU, %d host workers" % best},
        "step_seconds": [round(t, 6) for t in t1],
        "plain_fp64": {"value": round(statistics.mean(t0), 6), "unit": "s"},
        "speedup_chosen_vs_plain": round(statistics.mean(t0) / statistics.mean(t1), 3),
        "workers_sweep_s": {str(k): round(v, 4) for k, v in tune.items()},
        "iterations": {"min": int(it.min()), "max": int(it.max()), "mean": round(float(it.mean()), 2)},
        "statuses_ok": int(np.sum(st == 0)),
        "sum_setup_ms": round(float(sms.sum()), 1), "sum_solve_ms": round(float(pms.sum()), 1),
        "note": "value = wall seconds for set-up and PCG of every problem of the batch (inputs resident in HBM); "
                "sum_* are the per-problem times, which overlap on the GPU",
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.oracle_leg is not None:
        oracle_leg(args)
    elif args.workload == "batch256" and args.impl == "ours":
        if rank == 0:
            run_batch(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
