"""Benchmark of the GPU interior-point solver (one JSON line on rank 0).

A step is one complete solve (initial point, then IPM iterations until the
termination tests pass at eps_feas = 1e-8) of the mixed-cone QP workload:
n = 2000, m = 6600 (500 zero, 3000 nonneg, 500 SOC(5), 100 exp, 100
pow(0.3) rows/cones), P = diag + rank 10, A with 10 nnz per column, built
from a planted optimum (seeded synthetic data).  Every step passes through
all rows of the per-iteration device path.

metric  IPM iterations per second (total iterations / device time), for the
        FP32-factor + FP64-refinement path; the FP64-factor path is measured
        in the same run and reported under "fp64_factor"; time-to-1e-8 of
        both under "time_to_tol_ms".
N > 1   independent replicas, one problem per GPU (weak scaling, no
        collective on the data path).

serving  the MPC request stream (10 000 QPs, horizon U{10..50}, states
        U{4..12}, inputs U{2..4}, stable random dynamics, boxes and one SOC
        per step) through the continuous-batching server: solves/s and
        p50/p99 latency (submit -> result readable) at Poisson arrivals, next
        to one-at-a-time solves (clr_setup + clr_solve + read-back + free per
        problem), under "serving".

--impl reference times the FP64 CPU oracle on the host cores instead.
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

METRIC = "IPM iterations/s to eps_feas=1e-8 (time-to-1e-8 in time_to_tol_ms)"
UNIT = "iter/s"
WORKLOAD = "mixed-cone QP n=2000 m=6600 (500 zero, 3000 nonneg, 500 SOC5, 100 exp, 100 pow0.3), P=diag+rank10"
FP64_PEAK_TFLOPS = 1.25            # GB300 FP64 (FFMA and DMMA), nominal
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2070 MHz
FLOW_DRAM_BYTES_FP32 = 17.800448e6 + 1.957632e6    # k_bf_flow<float>, mixed-cone QP (profiles/k_bf_flow_*)


def measured_peaks():
    """HBM copy GB/s and cuBLAS BF16 TFLOP/s measured on this GPU model (file
    beside this script), else the fallback figures of one earlier measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


# Cone kernels at stress shapes (inputs far larger than the 129 MB L2): per unit
# (nonneg row, SOC(5) cone, PSD(10) cone) the algorithmic bytes of each step =
# the vectors it must read plus those it must write, 8 B per entry:
#   scaling:  s, z in; packed -H block and the scaling point (lambda) out
#             (nonneg 16 + 8 + 8; SOC d: 16d + 8 d(d+1)/2 + 8(d+2) with w-bar, eta;
#              PSD k: 16 d_k + 8 d_k(d_k+1)/2 + 8 (2 k^2 + k) for R, R^-1, lambda)
#   step:     s, z, ds, dz in (32 B per row; the result is one scalar)
#   ds:       lambda, W (w or w-bar; R, R^-1 for PSD), ds_a, dz_a in, d_s out
CONE_STRESS = [("nonneg", 1 << 26, 1), ("soc", 1 << 22, 5), ("psd", 1 << 16, 55)]


def cone_bytes(family, k):
    d = k
    if family == "nonneg":
        return {"scaling": 32, "step": 32, "ds": 40}
    if family == "soc":
        return {"scaling": 16 * d + 4 * d * (d + 1) + 8 * (d + 2), "step": 32 * d, "ds": 8 * (5 * d + 1)}
    kk = 10
    return {"scaling": 16 * d + 4 * d * (d + 1) + 8 * (2 * kk * kk + kk), "step": 32 * d,
            "ds": 8 * (4 * d + 2 * kk * kk + kk)}


def run_cone_roofline(clr, W, peaks, reps=10, shift=0):
    out = {}
    for fam, count, d in CONE_STRESS:
        count >>= shift
        cones, s, z, ds, dz = W.cone_stress(7, fam, count)
        t = clr.clr_cones_time(cones, s, z, ds, dz, 1.0, reps)
        del s, z, ds, dz
        b = cone_bytes(fam, d)
        row = {"units": count, "unit": {"nonneg": "row", "soc": "SOC(5) cone", "psd": "PSD(10) cone"}[fam]}
        for step, key in (("scaling", "scaling_ms"), ("step", "step_ms"), ("ds", "combined_ds_ms")):
            ms = t[key]
            gbs = b[step] * count / (ms / 1e3) / 1e9
            row[step] = {"ms": ms, "bytes_per_unit": b[step], "achieved_gbs": gbs,
                         "frac": gbs / peaks["hbm_gbs"]}
        out[fam] = row
    out["peak_gbs"] = peaks["hbm_gbs"]
    out["peak_source"] = peaks["source"] + " HBM copy"
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--factor-bits", type=int, default=32, choices=[16, 32, 64])
    ap.add_argument("--ir-stop-ratio", type=float, default=5.0,
                    help="refinement stall test (0 = the paper's rule only: tolerance or T_max)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch kernels directly instead of replaying captured graphs (for per-kernel profiling)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-cone-roofline", action="store_true",
                    help="skip the cone kernels at stress shapes (2^26 nonneg rows, 2^22 SOC5, 2^16 PSD10)")
    ap.add_argument("--configs", action="store_true",
                    help="solve each synthetic configuration once (absolute times, statuses, errors) and exit")
    ap.add_argument("--paper-workloads", action="store_true",
                    help="solve the paper's benchmark classes once each (portfolio and Huber QPs, entropy "
                         "maximisation; FP64 and FP32 factors) and exit")
    ap.add_argument("--cone-only", action="store_true",
                    help="run only the cone kernels at the stress shapes and print their JSON (for profiling)")
    ap.add_argument("--cone-shift", type=int, default=0, help="divide the stress shapes by 2^shift")
    ap.add_argument("--serve-requests", type=int, default=10_000)
    ap.add_argument("--serve-bits", type=int, default=64, choices=[32, 64])
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(seed, iters=2):
    """The oracle, as it stands, on the host cores: a bounded sample of the
    workload (its first `iters` IPM iterations; setup time subtracted)."""
    code = r"""
import sys, time, json
sys.path.insert(0, %r)
import oracle
from paper_2412_19027_gb300 import workloads as W
prob = W.mixed_cone(%d)
t0 = time.perf_counter(); oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones, settings=dict(max_iter=0)); t1 = time.perf_counter()
r = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones, settings=dict(max_iter=%d)); t2 = time.perf_counter()
print(json.dumps(dict(iters=r.iterations, setup=t1 - t0, total=t2 - t1)))
""" % (ROOT, seed, iters)
    cores = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS=str(cores), OPENBLAS_NUM_THREADS=str(cores), MKL_NUM_THREADS=str(cores))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    d = json.loads(out.stdout.strip().splitlines()[-1])
    t = max(d["total"] - d["setup"], 1e-9)
    return {"value": d["iters"] / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d IPM iterations of the same workload (FP64 NumPy/LAPACK oracle, dense KKT "
                      "8600x8600), setup time subtracted; %.1f s of CPU work" % (d["iters"], d["total"])}


def _pct(v, q):
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


def serve_stream(clr, sv, reqs, rate):
    """Submit reqs at Poisson arrivals of the given rate (per s; None = all at
    once) from a thread, wait for every result; latencies measured by the
    server (submit -> result readable)."""
    rng = np.random.default_rng(12345)
    gaps = rng.exponential(1.0 / rate, len(reqs)) if rate else np.zeros(len(reqs))
    arrivals = np.cumsum(gaps) - gaps[0]
    tickets = [None] * len(reqs)
    ready = threading.Event()

    def submitter():
        t0 = time.perf_counter()
        for k, r in enumerate(reqs):
            ta = t0 + arrivals[k]
            while True:
                d = ta - time.perf_counter()
                if d <= 0:
                    break
                if d > 2e-3:
                    time.sleep(d - 1e-3)
            tickets[k] = sv.submit(r)
            if k == 0:
                ready.set()
        ready.set()

    th = threading.Thread(target=submitter)
    t_start = time.perf_counter()
    th.start()
    lat, iters, statuses, unsolved = [], [], {}, []
    for k in range(len(reqs)):
        while tickets[k] is None:
            time.sleep(1e-4)
        res = sv.wait(tickets[k], 600.0)
        if res is None:
            raise RuntimeError("serving request timed out")
        info = res[3]
        lat.append(info["solve_s"])
        iters.append(info["iterations"])
        statuses[info["status_name"]] = statuses.get(info["status_name"], 0) + 1
        if info["status_name"] != "SOLVED" and len(unsolved) < 10:
            unsolved.append([k, info["status_name"], info["iterations"], info["fp64_from_iter"]])
    t_end = time.perf_counter()
    th.join()
    return {"requests": len(reqs), "offered_per_s": rate, "solves_per_s": len(reqs) / (t_end - t_start),
            "p50_ms": 1e3 * _pct(lat, 50), "p99_ms": 1e3 * _pct(lat, 99), "mean_iterations": float(np.mean(iters)),
            "statuses": statuses, "unsolved_first": unsolved}


def run_serving(args, clr, W):
    """The MPC request stream through the continuous-batching server, next to one-at-a-time solves."""
    t_gen = time.perf_counter()
    seeds = W.mpc_stream(args.seed, args.serve_requests)
    probs = [W.mpc_qp(sd) for sd in seeds]
    reqs = [clr.Request(p.P, p.q, p.A, p.b, p.cones) for p in probs]
    t_gen = time.perf_counter() - t_gen
    st = clr.clr_default_settings(args.serve_bits)
    # blocking parameters for the stream's cohorts, picked by the autotuner on a
    # 64-problem cohort of the stream's shapes (3 IPM iterations per candidate)
    t_tune = time.perf_counter()
    tune = clr.clr_autotune([(p.P, p.q, p.A, p.b, p.cones) for p in probs[-64:]], st, iters=3)
    tune["seconds"] = time.perf_counter() - t_tune
    st = clr.clr_default_settings(args.serve_bits, small_front_max=tune["small_front_max"],
                                  amalgamation=tune["amalgamation"], big_front_schedule=tune["big_front_schedule"])
    # one at a time: the whole public call sequence per problem
    k1 = min(200, len(probs))
    lat1 = []
    t0 = time.perf_counter()
    for p in probs[:k1]:
        a = time.perf_counter()
        s_ = clr.clr_setup(p.P, p.q, p.A, p.b, p.cones, st)
        s_.solve()
        s_.solution()
        s_.free()
        lat1.append(time.perf_counter() - a)
    rate1 = k1 / (time.perf_counter() - t0)
    one = {"solves_per_s": rate1, "p50_ms": 1e3 * _pct(lat1, 50), "p99_ms": 1e3 * _pct(lat1, 99),
           "sample": "first %d problems of the stream, sequential" % k1}
    sv = clr.Server(device_bytes=16 << 30, max_cohort=256, max_active=4, settings=st)
    serve_stream(clr, sv, reqs[:200], None)  # warm-up (pools, module load)
    sat = serve_stream(clr, sv, reqs, None)
    sat["arrivals"] = "all submitted at once (saturation)"
    pois = serve_stream(clr, sv, reqs, 0.8 * sat["solves_per_s"])
    pois["arrivals"] = "Poisson at 0.8 x saturation throughput"
    sweep = []
    for f in (0.25, 0.5, 0.8, 1.0, 1.2):
        nsw = int(min(500, len(reqs), max(50, 10.0 * f * rate1)))  # at most ~10 s per point
        r = serve_stream(clr, sv, reqs[:nsw], f * rate1)
        r["offered_x_one_at_a_time"] = f
        sweep.append(r)
    stats = sv.stats()
    sv.close()
    return {"workload": "MPC QP stream: %d requests, T U{10..50}, nx U{4..12}, nu U{2..4}, |x|<=5, |u|<=1, "
                        "||u_t||<=1.2, cost x'x + 0.1 u'u; FP%d factor" % (len(reqs), args.serve_bits),
            "server": {"max_cohort": 256, "max_active": 4, "device_budget_bytes": 16 << 30,
                       "cohorts": stats["cohorts"], "max_cohort_seen": stats["max_cohort_seen"],
                       "peak_device_bytes": stats["peak_bytes"]},
            "autotune": tune, "one_at_a_time": one, "saturation": sat, "poisson": pois,
            "sweep_vs_one_at_a_time": sweep,
            "speedup_solves_per_s": sat["solves_per_s"] / rate1, "generation_s": t_gen}


def run_paper_workloads(args, clr, W):
    """The paper's benchmark classes (Sec. 5.1 portfolio and Huber QPs, Sec. 5.3
    entropy maximisation), one timed solve per factor precision, setup reported
    apart.  Sizes below the paper's (n = 5000 / 5000 / 2000 there): at those the
    host setup of this solver takes 2.6 s (portfolio), 40 s (entropy) and 163 s
    (Huber: the ordering and the per-entry extend-add lists of fronts with thousands
    of children), so the smaller instances keep the run to a minute."""
    import torch

    out = {}
    for name, prob in (("portfolio_n2000", W.portfolio_qp(args.seed, n=2000)),
                       ("huber_n1000", W.huber_qp(args.seed, n=1000)),
                       ("entropy_n600", W.entropy_max(args.seed, n=600))):
        runs = []
        for bits in (64, 32):
            st = clr.clr_default_settings(bits)
            t0 = time.perf_counter()
            s_ = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
            t1 = time.perf_counter()
            s_.solve()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            x, _, _, info = s_.solution()
            pf = s_.perf()
            sym = s_.symbolic_stats()
            s_.free()
            runs.append({"factor_bits": bits, "status": info["status_name"], "iterations": info["iterations"],
                         "setup_s": t1 - t0, "solve_ms": 1e3 * (t2 - t1),
                         "factor_ms_per_factorization": pf["factor_ms"] / max(1, pf["factorizations"]),
                         "fp64_from_iter": info["fp64_from_iter"], "gap_rel": info["gap_rel"],
                         "res_primal": info["res_primal"], "res_dual": info["res_dual"],
                         "objective": float(prob.objective(x)), "kkt_dim": sym["kkt_dim"],
                         "l_nnz": sym["l_nnz"], "factor_flops": sym["factor_flops"], "max_front": sym["max_front"]})
        out[name] = runs
    return out


def run_configs(args, clr, W):
    """One timed solve of each configuration (setup reported apart), FP64 and the
    low-precision factors where the configuration asks for them."""
    import torch

    def one(prob, bits, **kw):
        st = clr.clr_default_settings(bits, **kw)
        t0 = time.perf_counter()
        s_ = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
        t1 = time.perf_counter()
        s_.solve()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        x, _, _, info = s_.solution()
        pf = s_.perf()
        sym = s_.symbolic_stats()
        s_.free()
        rec = {"factor_bits": bits, "status": info["status_name"], "iterations": info["iterations"],
               "setup_s": t1 - t0, "solve_ms": 1e3 * (t2 - t1),
               "device_ms": pf["init_ms"] + pf["resid_cones_ms"] + pf["factor_ms"] + pf["solve_step_ms"],
               "factor_ms_per_factorization": pf["factor_ms"] / max(1, pf["factorizations"]),
               "ir_steps_total": info["ir_steps_total"], "fp64_from_iter": info["fp64_from_iter"],
               "res_primal": info["res_primal"], "res_dual": info["res_dual"], "gap_rel": info["gap_rel"],
               "kkt_dim": sym["kkt_dim"], "l_nnz": sym["l_nnz"], "factor_flops": sym["factor_flops"],
               "max_front": sym["max_front"]}
        if getattr(prob, "x_star", None) is not None:
            f_star = prob.objective(prob.x_star)
            rec["objective_rel_err_vs_planted"] = abs(prob.objective(x) - f_star) / max(1.0, abs(f_star))
        return rec

    out = {}
    p0 = W.nonneg_qp(args.seed)
    out["qp_nonneg_n50_m100"] = [one(p0, 64)]
    # throughput: a cohort of 4096 seeds of the same shape in one solver
    probs = [W.nonneg_qp(args.seed + k) for k in range(4096)]
    st = clr.clr_default_settings(64)
    t0 = time.perf_counter()
    bt = clr.clr_batch_setup([(p.P, p.q, p.A, p.b, p.cones) for p in probs], st)
    t1 = time.perf_counter()
    bt.solve()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    stats = {}
    for k in range(len(probs)):
        nm = bt.info_of(k)["status_name"]
        stats[nm] = stats.get(nm, 0) + 1
    bt.free()
    out["qp_nonneg_n50_m100_cohort4096"] = {"setup_s": t1 - t0, "solve_ms": 1e3 * (t2 - t1),
                                            "solves_per_s": len(probs) / (t2 - t1), "statuses": stats}
    out["mixed_n2000_m6600"] = [one(W.mixed_cone(args.seed), b, ir_stop_ratio=5.0) for b in (64, 32, 16)]
    pc2 = W.banded_lp(args.seed)
    out["banded_n200000_m400000"] = [one(pc2, b, ir_stop_ratio=5.0) for b in (64, 32, 16)]
    pc3 = W.psd_batch(args.seed)
    out["psd2000x10_n20000"] = [one(pc3, b, ir_stop_ratio=5.0) for b in (32, 64)]
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    iters_per_step = 1
    sample_times = []
    code_iters = 0
    import oracle
    from paper_2412_19027_gb300 import workloads as W
    prob = W.mixed_cone(args.seed)
    t0 = time.perf_counter()
    oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones, settings=dict(max_iter=0))
    setup = time.perf_counter() - t0
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        r = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones, settings=dict(max_iter=iters_per_step))
        dt = time.perf_counter() - t - setup
        if k >= args.warmup:
            sample_times.append(max(dt, 1e-9))
            code_iters += r.iterations
    total = sum(sample_times)
    value = code_iters / total
    cores = os.cpu_count() or 1
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "seed": args.seed,
                       "step": "one IPM iteration of the oracle (bounded sample of the solve)"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                             "sample": "%d steps x %d IPM iteration(s), setup subtracted" % (args.steps,
                                                                                            iters_per_step)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2412_19027_gb300 import build as B
    if rank == 0:
        B.build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_2412_19027_gb300 import clr, workloads as W
    if args.configs:
        if rank == 0:
            print(json.dumps({"configs": run_configs(args, clr, W)}), flush=True)
        return
    if args.paper_workloads:
        if rank == 0:
            print(json.dumps({"paper_workloads": run_paper_workloads(args, clr, W)}), flush=True)
        return
    if args.cone_only:
        if rank == 0:
            print(json.dumps({"cone_roofline": run_cone_roofline(clr, W, measured_peaks(), 3, args.cone_shift)}),
                  flush=True)
        return
    prob = W.mixed_cone(args.seed + rank)
    n, m = prob.n, prob.m
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2

    def make(bits):
        kw = {"ir_stop_ratio": args.ir_stop_ratio, "use_graph": 0 if args.no_graph else 1}
        st = clr.clr_default_settings(bits, **kw)
        s = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
        s.set_stream(stream.cuda_stream)
        return s

    def timed(solver, steps, warmup):
        for _ in range(warmup):
            solver.solve()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        iters, launches, perfs, infos = 0, 0, [], []
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                starts[k].record(stream)
            solver.solve()
            ends[k].record(stream)
            info = solver.info()
            p = solver.perf()
            iters += info["iterations"]
            launches += p["kernel_launches"]
            perfs.append(p)
            infos.append(info)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        times = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
        return times, iters, launches, perfs, infos

    main = make(args.factor_bits)
    sym = main.symbolic_stats()
    clocks = ClockSampler(local)
    clocks.start()
    times, iters, launches, perfs, infos = timed(main, args.steps, args.warmup)
    clk = clocks.stop()
    total_ms = float(sum(times))
    if ws > 1:
        t = torch.tensor([total_ms, float(iters)], device="cuda", dtype=torch.float64)
        tmax = t.clone()
        torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
        tsum = t.clone()
        torch.distributed.all_reduce(tsum, op=torch.distributed.ReduceOp.SUM)
        total_ms_max, iters_all = float(tmax[0]), float(tsum[1])
    else:
        total_ms_max, iters_all = total_ms, float(iters)
    value = iters_all / (total_ms_max / 1e3)
    x, s_, z, info = main.solution()
    f_star = prob.objective(prob.x_star)
    obj_err = abs(prob.objective(x) - f_star) / max(1.0, abs(f_star))

    # the FP64-factor path on the same problem
    fp64 = None
    if args.fp64_steps > 0:
        s64 = main if args.factor_bits == 64 else make(64)
        t64, it64, _, p64, inf64 = timed(s64, args.fp64_steps, 1)
        x64, _, _, _ = s64.solution()
        fp64 = {"time_to_tol_ms": float(np.median(t64)), "iterations": inf64[-1]["iterations"],
                "iters_per_s": it64 / (sum(t64) / 1e3), "status": inf64[-1]["status_name"],
                "objective_rel_err_vs_planted": abs(prob.objective(x64) - f_star) / max(1.0, abs(f_star)),
                "factor_ms_per_factorization": p64[-1]["factor_ms"] / max(1, p64[-1]["factorizations"])}
        if s64 is not main:
            s64.free()

    # end to end through the C ABI with host buffers: q, b in; x, s, z out
    e2e = None
    if not args.no_e2e:
        e_iters, e_time = 0, 0.0
        for k in range(args.steps):
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            main.update_qb(prob.q, prob.b)
            main.solve()
            xo, so, zo, info_e = main.solution()
            e_time += time.perf_counter() - t0
            e_iters += info_e["iterations"]
        e2e = {"value": e_iters / e_time, "unit": UNIT, "h2d_bytes_per_step": 8 * (n + m),
               "d2h_bytes_per_step": 8 * (n + 2 * m)}

    # dominant phase and its roofline
    p = perfs[-1]
    nf = max(1, p["factorizations"])
    phases = {"residuals+cones": p["resid_cones_ms"], "factorization": p["factor_ms"],
              "solves+steps": p["solve_step_ms"], "init": p["init_ms"]}
    fact_ms = p["factor_ms"] / nf
    peaks = measured_peaks()
    achieved = sym["factor_flops"] / (fact_ms / 1e3) / 1e12
    if args.factor_bits == 16:
        # BF16 products on the tensor cores, timed inside the solve: the sustained figure
        bound, peak = "tensor", peaks["bf16_tflops_sustained"]
        psrc = "%s cuBLAS BF16 sustained" % peaks["source"]
    elif args.factor_bits == 32:
        bound, peak, psrc = "alu", FP32_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"
    else:
        bound, peak, psrc = "alu", FP64_PEAK_TFLOPS, "GB300 FP64 nominal 1.25 TFLOP/s"
    # DRAM bytes of the factorization's dominant launch (k_bf_flow, one per factorization
    # of this workload) from one ncu capture of this kernel version (profiles/); other
    # precisions were not captured
    traffic = FLOW_DRAM_BYTES_FP32 if (args.factor_bits == 32 and not args.no_graph) else None
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "numeric LDL^T (multifrontal, FP%d)" % args.factor_bits,
                "flops_per_launch": sym["factor_flops"], "ms_per_launch": fact_ms, "peak_source": psrc,
                "traffic_source": "ncu dram__bytes_read+write of k_bf_flow<float> (dominant launch)" if traffic
                else None}
    cone_roof = None
    if not args.no_cone_roofline and rank == 0:
        cone_roof = run_cone_roofline(clr, W, peaks)

    serving = None
    if not args.no_serving:
        serving = run_serving(args, clr, W)

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            try:
                cpu = cpu_baseline(args.seed)
            except Exception as e:  # the baseline is informative only
                cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                       "sample": "failed: %s" % str(e)[:200]}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64 (f%d factor)" % args.factor_bits, "data": "synthetic",
                "config": {"workload": WORKLOAD, "seed": args.seed, "factor_bits": args.factor_bits,
                           "eps_feas": 1e-8, "l2": "flushed (256 MB write) before every timed solve",
                           "parallelism": "replicas" if ws > 1 else "single GPU",
                           "ir_stop_ratio": main.settings.ir_stop_ratio, "cuda_graphs": not args.no_graph},
                "time_to_tol_ms": {"median": float(np.median(times)), "fp64_factor": fp64["time_to_tol_ms"] if fp64
                                   else None},
                "iterations": infos[-1]["iterations"], "status": infos[-1]["status_name"],
                "objective_rel_err_vs_planted": obj_err, "res_primal": infos[-1]["res_primal"],
                "res_dual": infos[-1]["res_dual"], "ir_steps_total": infos[-1]["ir_steps_total"],
                "fp64_from_iter": infos[-1]["fp64_from_iter"], "fp64_factor": fp64, "phase_ms_per_solve": phases, "roofline": roofline,
                "gpu_launches": int(launches), "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
                "serving": serving, "cone_roofline": cone_roof,
                "symbolic": {k: sym[k] for k in ("kkt_dim", "l_nnz", "factor_flops", "n_supernodes", "n_levels",
                                                 "max_front")}}
        print(json.dumps(line), flush=True)
    main.free()
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
