"""Benchmark of the GPU interior-point solver (one JSON line on rank 0).

Workload: the large sparse LP (banded LP) n = 200 000, m = 400 000: 100 000
zero-cone and 300 000 nonnegative rows, A with 8 N(0,1) entries per column
(6 band rows around 2j plus 2 rows uniform in a window of 1024), P diagonal
U(0,1) with half of it zero, built from a planted optimum (seeded synthetic
data).  eps_feas = 1e-8.

step    one IPM iteration of Algorithm 1 (residuals, termination tests, cone
        scalings, KKT factorization, the three refined KKT solves, step
        lengths, combined direction, update: every row of the per-iteration
        device step), run through clr_solve_iterate on the solver's stream;
        the timed region starts a fresh solve (its initial point included) and
        starts another one whenever a solve ends inside it.
metric  IPM iterations per second of the FP32-factor + FP64-refinement path
        (with its escalation to the FP64 factor); time-to-1e-8 of full solves
        with the FP32 factor, the FP64 factor and the 16-bit-product factor,
        each with its error against the planted optimum, under
        "time_to_tol_ms".
N > 1   independent replicas, one problem per GPU (weak scaling, no
        collective on the data path).

Also reported: the mixed-cone QP (n = 2000, m = 6600) under "mixed_cone_qp";
the MPC serving stream (FP64 and FP32 factors) under "serving"; the cone
kernels at stress shapes under "cone_roofline"; the GPU's measured
arithmetic peaks (the library's probe) under "peaks".

--impl reference times the FP64 CPU oracle on the host cores instead (one IPM
iteration per step on a scaled-down instance of the same generator: the dense
oracle cannot hold the full KKT matrix of order 600 000).
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

METRIC = "IPM iterations/s to eps_feas=1e-8 (time-to-1e-8 of the FP32, FP64 and 16-bit-product factors in time_to_tol_ms)"
UNIT = "iter/s"
WORKLOAD = ("banded LP n=200000 m=400000 (100000 zero, 300000 nonneg rows), A 8 nnz/col (6 band + 2 in a "
            "1024 window), P diag U(0,1) half zero, planted optimum")
SAMPLE_N = 2000  # scaled-down instance of the same generator for the CPU oracle (dense KKT of order 6000)


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


# FP64 flops per unit of each cone step, counted from the kernel sources (an FMA as
# 2 flops, a square root or a division as 1, which favours the kernels: on a GB300
# they cost several FMA slots each).  nonneg: lambda = sqrt(s z), w = s / lambda,
# H = w^2; step: two ratios; d_s: the Jordan product, quotient and scaling.  SOC(5):
# J-norms, gamma, eta, w-bar, lambda and the 15 packed H entries; step: both
# quadratic root tests; d_s: W^{-1} ds_a, W dz_a, their Jordan product, the
# quotient by lambda, W.  PSD(10): two 10 x 10 Cholesky factors, L_z^T L_s,
# a one-sided Jacobi SVD (about 6 sweeps), R, R^{-1} and the 55 x 55 packed H;
# step: per side a Cholesky, L^{-1} dS L^{-T}, a Householder tridiagonalisation
# and about 48 Sturm counts of the bisection (4 flops per row each); d_s:
# congruences with R, R^{-1}.
CONE_FP64_FLOPS = {"nonneg": {"scaling": 4, "step": 4, "ds": 8},
                   "soc": {"scaling": 150, "step": 80, "ds": 100},
                   "psd": {"scaling": 30_000, "step": 11_000, "ds": 8_000}}


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
            if peaks.get("fp64_tflops"):
                fl = CONE_FP64_FLOPS[fam][step]
                tf = fl * count / (ms / 1e3) / 1e12
                row[step].update({"fp64_flops_per_unit": fl, "achieved_fp64_tflops": tf,
                                  "frac_fp64": tf / peaks["fp64_tflops"]})
        out[fam] = row
    out["peak_gbs"] = peaks["hbm_gbs"]
    out["peak_source"] = peaks["source"] + " HBM copy"
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed IPM iterations")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--factor-bits", type=int, default=32, choices=[16, 32, 64])
    ap.add_argument("--n", type=int, default=0, help="banded LP size (default: the full n=200000)")
    ap.add_argument("--ir-stop-ratio", type=float, default=5.0,
                    help="refinement stall test (0 = the paper's rule only: tolerance or T_max)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch kernels directly instead of replaying captured graphs (for per-kernel profiling)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--fp64-steps", type=int, default=1, help="0 skips the FP64 and 16-bit full solves")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-cone QP leg")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-tc-factor", action="store_true",
                    help="skip the FP32 factorization of the batched PSD problem with and without tensor cores")
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
    ap.add_argument("--init-only", action="store_true",
                    help="set up the workload (--n, --factor-bits, --no-graph) and run only the initial point "
                         "(one factorization and its solves), then exit: the case the factorization profiles use")
    ap.add_argument("--init-workload", default="banded_lp", choices=["banded_lp", "psd_batch"],
                    help="--init-only: the banded LP of order --n, or the PSD batch with n = --n variables, "
                         "n/10 PSD(10) cones and n/4 nonnegative rows")
    ap.add_argument("--big-front-schedule", type=int, default=1, choices=[0, 1, 2, 3],
                    help="large-front schedule of every solve (the setting of that name)")
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
    workload -- its first `iters` IPM iterations on the same generator at
    n = SAMPLE_N (the dense oracle cannot hold the full problem), setup time
    subtracted."""
    code = r"""
import sys, time, json
sys.path.insert(0, %r)
import oracle
from paper_2412_19027_gb300 import workloads as W
prob = W.banded_lp(%d, n=%d)
t0 = time.perf_counter(); oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones, settings=dict(max_iter=0)); t1 = time.perf_counter()
r = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones, settings=dict(max_iter=%d)); t2 = time.perf_counter()
print(json.dumps(dict(iters=r.iterations, setup=t1 - t0, total=t2 - t1)))
""" % (ROOT, seed, SAMPLE_N, iters)
    cores = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS=str(cores), OPENBLAS_NUM_THREADS=str(cores), MKL_NUM_THREADS=str(cores))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    d = json.loads(out.stdout.strip().splitlines()[-1])
    t = max(d["total"] - d["setup"], 1e-9)
    return {"value": d["iters"] / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "first %d IPM iterations of the same generator at n=%d, m=%d (FP64 NumPy/LAPACK oracle, dense "
                      "KKT of order %d), setup time subtracted; %.1f s of CPU work" % (
                          d["iters"], SAMPLE_N, 2 * SAMPLE_N, 3 * SAMPLE_N, d["total"])}


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


def make_stream(args, clr, W):
    t_gen = time.perf_counter()
    seeds = W.mpc_stream(args.seed, args.serve_requests)
    probs = [W.mpc_qp(sd) for sd in seeds]
    reqs = [clr.Request(p.P, p.q, p.A, p.b, p.cones) for p in probs]
    return probs, reqs, time.perf_counter() - t_gen


def run_serving(args, clr, W, bits, stream, sweep_points=(0.25, 0.5, 0.8, 1.0, 1.2), k_one=200):
    """The MPC request stream through the continuous-batching server, next to one-at-a-time solves."""
    probs, reqs, t_gen = stream
    st = clr.clr_default_settings(bits)
    # blocking parameters for the stream's cohorts, picked by the autotuner on a
    # 64-problem cohort of the stream's shapes (3 IPM iterations per candidate)
    t_tune = time.perf_counter()
    tune = clr.clr_autotune([(p.P, p.q, p.A, p.b, p.cones) for p in probs[-64:]], st, iters=3)
    tune["seconds"] = time.perf_counter() - t_tune
    st = clr.clr_default_settings(bits, small_front_max=tune["small_front_max"],
                                  amalgamation=tune["amalgamation"], big_front_schedule=tune["big_front_schedule"])
    # one at a time: the whole public call sequence per problem
    k1 = min(k_one, len(probs))
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
    for f in sweep_points:
        nsw = int(min(500, len(reqs), max(50, 10.0 * f * rate1)))  # at most ~10 s per point
        r = serve_stream(clr, sv, reqs[:nsw], f * rate1)
        r["offered_x_one_at_a_time"] = f
        sweep.append(r)
    stats = sv.stats()
    sv.close()
    return {"workload": "MPC QP stream: %d requests, T U{10..50}, nx U{4..12}, nu U{2..4}, |x|<=5, |u|<=1, "
                        "||u_t||<=1.2, cost x'x + 0.1 u'u; FP%d factor" % (len(reqs), bits),
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
    """The oracle on the host cores, on the same generator at n = SAMPLE_N: one
    IPM iteration per step (the dense oracle cannot hold the full problem)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2412_19027_gb300 import workloads as W
    prob = W.banded_lp(args.seed, n=SAMPLE_N)
    t0 = time.perf_counter()
    oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones, settings=dict(max_iter=0))
    setup = time.perf_counter() - t0
    sample_times, code_iters = [], 0
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        r = oracle.solve(prob.P, prob.q, prob.A, prob.b, prob.cones, settings=dict(max_iter=1))
        dt = time.perf_counter() - t - setup
        if k >= args.warmup:
            sample_times.append(max(dt, 1e-9))
            code_iters += r.iterations
    total = sum(sample_times)
    value = code_iters / total
    cores = os.cpu_count() or 1
    sample = ("%d steps x 1 IPM iteration of the same generator at n=%d, m=%d (dense KKT of order %d), setup "
              "subtracted" % (args.steps, SAMPLE_N, 2 * SAMPLE_N, 3 * SAMPLE_N))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "seed": args.seed,
                       "step": "one IPM iteration of the oracle on the scaled-down instance (bounded sample)"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT, "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _events(torch, n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def timed_solves(torch, solver, stream, flush, count):
    """`count` full solves (clr_solve) timed with CUDA events on the solver's
    stream, L2 flushed before each; returns (ms list, info of the last, perf of the last)."""
    st, en = _events(torch, count), _events(torch, count)
    out, info, perf = [], None, None
    for k in range(count):
        with torch.cuda.stream(stream):
            flush.zero_()
            st[k].record(stream)
        solver.solve()
        en[k].record(stream)
        info, perf = solver.info(), solver.perf()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(st, en)], info, perf


def factor_roofline(perf, sym, peaks):
    """Roofline of the numeric factorization, per precision it ran in during the
    solve: unit = one factorization (all launches of the factorization phase),
    algorithmic flops = the symbolic factor flop count, time = CUDA events around
    the phase inside the captured iteration graphs."""
    out = {}
    n64 = perf["factorizations64"]
    f64_ms = perf["factor64_ms"]
    f32_ms = perf["factor_ms"] - f64_ms
    # factorizations of the iterations (redone iterations included); the
    # initial-point factorization (one for problems of symmetric cones only, as
    # here) is timed in init_ms and left out
    n32 = max(0, perf["factorizations"] - n64 - 1)
    for name, n, ms, peak, src in (("fp32", n32, f32_ms, peaks["fp32_fma_tflops"], "measured FP32 FMA (library probe)"),
                                   ("fp64", n64, f64_ms, peaks["fp64_fma_tflops"], "measured FP64 FMA (library probe)")):
        if n <= 0 or ms <= 0:
            continue
        per = ms / n
        ach = sym["factor_flops"] / (per / 1e3) / 1e12
        out[name] = {"factorizations": n, "ms_per_factorization": per, "total_ms": ms, "achieved_tflops": ach,
                     "peak_tflops": peak, "peak_source": src, "frac": ach / peak}
    return out


def solve_roofline(perf, info, sym, peaks):
    """The solve phase (refined KKT solves, direction recovery, step lengths,
    update): unit = one KKT solve (a forward and a backward sweep over the factor);
    algorithmic bytes = 2 nnz(L) x the factor's element size (each sweep reads the
    factor once; vectors are O(N) and left out); solves = 3 per iteration + the
    refinement steps (the initial point's are in init_ms); time = the phase's CUDA
    events, so the other work of the phase is charged to the solves."""
    n64 = perf["factorizations64"]
    n_all = max(1, perf["factorizations"] - 1)
    w = (8.0 * n64 + 4.0 * (n_all - n64)) / n_all if n_all else 8.0
    solves = 3 * info["iterations"] + info["ir_steps_total"]
    if solves <= 0 or perf["solve_step_ms"] <= 0:
        return None
    per = perf["solve_step_ms"] / solves
    byts = 2.0 * sym["l_nnz"] * w
    gbs = byts / (per / 1e3) / 1e9
    return {"solves": solves, "ms_per_solve": per, "bytes_per_solve": byts, "achieved_gbs": gbs,
            "peak_gbs": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"], "bound": "hbm",
            "note": "factor element size averaged over the iterations' FP32 / FP64 factors"}


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
    if args.init_only:
        if rank == 0:
            if args.init_workload == "psd_batch":
                nn = args.n or 20000
                prob = W.psd_batch(args.seed, n=nn, n_psd=nn // 10, n_nonneg=nn // 4)
            else:
                prob = W.banded_lp(args.seed, n=args.n) if args.n else W.banded_lp(args.seed)
            st = clr.clr_default_settings(args.factor_bits, ir_stop_ratio=args.ir_stop_ratio, max_iter=0,
                                          use_graph=0 if args.no_graph else 1,
                                          big_front_schedule=args.big_front_schedule)
            s_ = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
            s_.solve()
            info, sym = s_.info(), s_.symbolic_stats()
            s_.free()
            print(json.dumps({"init_only": {"status": info["status_name"], "kkt_dim": sym["kkt_dim"],
                                            "l_nnz": sym["l_nnz"], "n_levels": sym["n_levels"]}}), flush=True)
        return
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    peaks = clr.clr_probe_peaks(5, stream.cuda_stream)
    copy_peaks = measured_peaks()
    peaks.update({"hbm_gbs": copy_peaks["hbm_gbs"], "bf16_cublas_tflops": copy_peaks["bf16_tflops"],
                  "hbm_source": copy_peaks["source"] + " (MEASURED_PEAKS.json copy test)"})

    t_gen = time.perf_counter()
    prob = W.banded_lp(args.seed + rank, n=args.n) if args.n else W.banded_lp(args.seed + rank)
    t_gen = time.perf_counter() - t_gen
    n, m = prob.n, prob.m
    f_star = prob.objective(prob.x_star)

    def make(bits):
        kw = {"ir_stop_ratio": args.ir_stop_ratio, "use_graph": 0 if args.no_graph else 1,
              "big_front_schedule": args.big_front_schedule}
        st = clr.clr_default_settings(bits, **kw)
        t0 = time.perf_counter()
        s = clr.clr_setup(prob.P, prob.q, prob.A, prob.b, prob.cones, st)
        s.set_stream(stream.cuda_stream)
        return s, time.perf_counter() - t0

    def err_of(x):
        return abs(prob.objective(x) - f_star) / max(1.0, abs(f_star))

    # ---------------- headline: IPM iterations, FP32 factor + FP64 refinement
    main, setup_s = make(args.factor_bits)
    sym = main.symbolic_stats()
    main.solve_begin()
    for _ in range(args.warmup):
        done, _ = main.solve_iterate(1)
        if done:
            main.solve_end()
            main.solve_begin()
    main.solve_end()
    starts, ends = _events(torch, args.steps), _events(torch, args.steps)
    iters, restarts = 0, 0
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            starts[k].record(stream)
        if k == 0:
            main.solve_begin()  # a fresh solve: its initial point is inside the timed region
        done, ran = main.solve_iterate(1)
        iters += ran
        if done:
            main.solve_end()
            main.solve_begin()
            restarts += 1
        ends[k].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    main.solve_end()
    times = [a.elapsed_time(b) for a, b in zip(starts, ends)]
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

    # ---------------- time to 1e-8: full solves in each factor precision
    ttt = {}
    t32, inf32, pf32 = timed_solves(torch, main, stream, flush, 2)
    x32, _, _, _ = main.solution()
    ttt["fp32_factor"] = {"ms": float(np.median(t32)), "all_ms": t32, "iterations": inf32["iterations"],
                          "status": inf32["status_name"], "fp64_from_iter": inf32["fp64_from_iter"],
                          "objective_rel_err_vs_planted": err_of(x32), "gap_rel": inf32["gap_rel"],
                          "res_primal": inf32["res_primal"], "res_dual": inf32["res_dual"],
                          "ir_steps_total": inf32["ir_steps_total"], "setup_s": setup_s,
                          "phase_ms": {"init": pf32["init_ms"], "residuals+cones": pf32["resid_cones_ms"],
                                       "factorization": pf32["factor_ms"], "solves+steps": pf32["solve_step_ms"]},
                          "factorization_roofline": factor_roofline(pf32, sym, peaks),
                          "solve_roofline": solve_roofline(pf32, inf32, sym, peaks)}
    # end to end through the C ABI with host buffers: q, b in; x, s, z out (one full solve per step)
    e2e = None
    if not args.no_e2e:
        e_iters, e_time = 0, 0.0
        for k in range(args.e2e_steps):
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
               "d2h_bytes_per_step": 8 * (n + 2 * m),
               "step": "one full solve through the public API (clr_update_qb from host q, b; clr_solve; "
                       "clr_get_solution to host x, s, z); %d solves" % args.e2e_steps}
    main.free()
    for bits, key in ((64, "fp64_factor"), (16, "bf16_products_fp32_factor")):
        if args.fp64_steps <= 0:
            break
        sv_, su = make(bits)
        tt, inf, pf = timed_solves(torch, sv_, stream, flush, 1)
        xx, _, _, _ = sv_.solution()
        ttt[key] = {"ms": float(np.median(tt)), "iterations": inf["iterations"], "status": inf["status_name"],
                    "fp64_from_iter": inf["fp64_from_iter"], "objective_rel_err_vs_planted": err_of(xx),
                    "gap_rel": inf["gap_rel"], "res_primal": inf["res_primal"], "res_dual": inf["res_dual"],
                    "ir_steps_total": inf["ir_steps_total"], "setup_s": su,
                    "phase_ms": {"init": pf["init_ms"], "residuals+cones": pf["resid_cones_ms"],
                                 "factorization": pf["factor_ms"], "solves+steps": pf["solve_step_ms"]},
                    "factorization_roofline": factor_roofline(pf, sym, peaks),
                    "solve_roofline": solve_roofline(pf, inf, sym, peaks)}
        sv_.free()
    if "fp64_factor" in ttt:
        ttt["fp32_speedup_vs_fp64_factor"] = ttt["fp64_factor"]["ms"] / ttt["fp32_factor"]["ms"]

    # dominant kernel of the headline solve: the factorization phase in the
    # precision that took the most time
    fr = ttt["fp32_factor"]["factorization_roofline"]
    dom = max(fr.items(), key=lambda kv: kv[1]["total_ms"]) if fr else None
    roofline = None
    if dom:
        name, d = dom
        roofline = {"bound": "alu", "achieved": d["achieved_tflops"], "peak": d["peak_tflops"], "unit": "TFLOP/s",
                    "frac": d["frac"], "traffic": None,
                    "kernel": "numeric LDL^T, %s factor (k_bf_flow dataflow launches + small-front kernels of one "
                              "factorization)" % name.upper(),
                    "flops_per_launch": sym["factor_flops"], "ms_per_launch": d["ms_per_factorization"],
                    "peak_source": d["peak_source"] + ", of measured",
                    "unit_of_launch": "one numeric factorization of the KKT matrix (order %d)" % sym["kkt_dim"],
                    "traffic_source": "not captured for this kernel version"}

    # ---------------- the mixed-cone QP (earlier headline workload)
    mixed = None
    if not args.no_mixed and rank == 0:
        pm = W.mixed_cone(args.seed)
        mixed = {}
        for bits in (32, 64):
            st = clr.clr_default_settings(bits, ir_stop_ratio=args.ir_stop_ratio)
            sv_ = clr.clr_setup(pm.P, pm.q, pm.A, pm.b, pm.cones, st)
            sv_.set_stream(stream.cuda_stream)
            sv_.solve()
            tt, inf, pf = timed_solves(torch, sv_, stream, flush, 3)
            xx, _, _, _ = sv_.solution()
            fs = pm.objective(pm.x_star)
            mixed["fp%d_factor" % bits] = {"time_to_tol_ms": float(np.median(tt)), "iterations": inf["iterations"],
                                           "status": inf["status_name"], "fp64_from_iter": inf["fp64_from_iter"],
                                           "objective_rel_err_vs_planted": abs(pm.objective(xx) - fs) / max(1.0, abs(fs)),
                                           "factor_ms_per_factorization": pf["factor_ms"] / max(1, pf["factorizations"])}
            sv_.free()
        mixed["workload"] = "mixed-cone QP n=2000 m=6600 (500 zero, 3000 nonneg, 500 SOC5, 100 exp, 100 pow0.3), P=diag+rank10"

    # ---------------- the FP32 factorization with tensor-core updates: the batched
    # PSD problem (its large fronts are throughput-bound, so the per-level choice
    # puts them on the tensor cores) against the CUDA-core launch
    tcf = None
    if not args.no_tc_factor and rank == 0:
        pp = W.psd_batch(args.seed)
        tcf = {"workload": "batched PSD problem n=20000: 2000 PSD(10) cones + 5000 nonneg rows, P=0 (FP32 factor)"}
        for sched, key in ((1, "tensor_cores_where_chosen"), (2, "cuda_cores")):
            st = clr.clr_default_settings(32, ir_stop_ratio=args.ir_stop_ratio, max_iter=2, big_front_schedule=sched)
            t0 = time.perf_counter()
            sv_ = clr.clr_setup(pp.P, pp.q, pp.A, pp.b, pp.cones, st)
            su = time.perf_counter() - t0
            sv_.set_stream(stream.cuda_stream)
            sv_.solve()
            _, _, pf = timed_solves(torch, sv_, stream, flush, 2)
            sy_ = sv_.symbolic_stats()
            sv_.free()
            ms = pf["factor_ms"] / max(1, pf["factorizations"])
            tf = sy_["factor_flops"] / (ms * 1e-3) / 1e12
            tcf[key] = {"ms_per_factorization": ms, "factorizations": pf["factorizations"],
                        "achieved_tflops": tf, "factor_flops": sy_["factor_flops"], "setup_s": su,
                        "frac_of_tf32_tensor_peak": tf / peaks["tf32_tc_tflops"],
                        "frac_of_fp32_fma_peak": tf / peaks["fp32_fma_tflops"]}
        tcf["speedup"] = tcf["cuda_cores"]["ms_per_factorization"] / tcf["tensor_cores_where_chosen"]["ms_per_factorization"]
        tcf["note"] = ("flops = the LDL^T's exact symbolic count per factorization; each 64 x 64 x 64 tile update "
                       "issues 4x its flops as TF32 MMAs (high and low parts of both operands), so the algorithmic "
                       "rate is bounded by 1/4 of the TF32 peak")

    cone_roof = None
    if not args.no_cone_roofline and rank == 0:
        cone_roof = run_cone_roofline(clr, W, {"hbm_gbs": peaks["hbm_gbs"], "source": copy_peaks["source"],
                                               "fp64_tflops": peaks["fp64_fma_tflops"]})
        cone_roof["fp64_peak_tflops"] = peaks["fp64_fma_tflops"]
        cone_roof["fp64_peak_source"] = "measured FP64 FMA (library probe)"

    serving = None
    if not args.no_serving:
        stream_reqs = make_stream(args, clr, W)
        serving = {"fp64_factor": run_serving(args, clr, W, 64, stream_reqs),
                   "fp32_factor": run_serving(args, clr, W, 32, stream_reqs, sweep_points=(0.8,), k_one=100)}

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
                           "eps_feas": 1e-8, "step": "one IPM iteration (clr_solve_iterate); the timed region "
                           "starts a fresh solve and restarts one whenever a solve ends",
                           "l2": "flushed (256 MB write) before every timed step; the KKT factor (%.0f MB) is "
                                 "larger than L2 as well" % (sym["l_nnz"] * 4 / 1e6),
                           "parallelism": "replicas" if ws > 1 else "single GPU",
                           "ir_stop_ratio": args.ir_stop_ratio, "cuda_graphs": not args.no_graph,
                           "escalate_ratio": 0.1},
                "iterations_timed": iters, "solves_restarted_in_timed_region": restarts,
                "time_to_tol_ms": ttt, "roofline": roofline, "peaks": peaks,
                "gpu_launches": int(pf32["kernel_launches"] * iters / max(1, pf32["iterations"])),
                "gpu_launches_note": "kernels per timed region, from the solver's count per full solve scaled by "
                                     "the iterations timed",
                "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
                "mixed_cone_qp": mixed, "serving": serving, "cone_roofline": cone_roof,
                "tensor_core_factorization": tcf,
                "generation_s": t_gen,
                "symbolic": {k: sym[k] for k in ("kkt_dim", "l_nnz", "factor_flops", "n_supernodes", "n_levels",
                                                 "max_front")}}
        print(json.dumps(line), flush=True)
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
