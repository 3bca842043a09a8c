"""Benchmark: batched NLL + gradient evaluations per second on one GB300.

Workload (the batched pseudo-experiment configuration): T toys of the
two-dataset generalized-gamma workload -- 16 species on a 20000-point fine
grid (0.1 keV, 0-2 MeV), 2 datasets (exposures 1.0 / 0.6) on a 1200-bin
domain of 1 p.e. bins, 23 parameters, two pulls.  Toy t has Poisson counts
drawn from the stored expected counts at theta0 (seed 1000 + t), its own
parameter vector theta0 (1 + 0.01 N(0,1)) and a fit window of 600..1200 bins.
One step = one NLL + gradient evaluation of every toy (column prologue,
response build + contraction, FP64 deviance and reduction, adjoint, gradient
reduction) in the mixed-precision path; inputs resident in HBM.

Under torchrun each rank evaluates its own T toys (weak scaling, no collective
on the data path; only the timing uses a barrier and a max over ranks).
`--impl reference` times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NLL+grad evals/sec (batched toys) on 1 GB300, mixed vs FP64 path at |dNLL|<1e-3"
UNIT = "evals/s"
WORKLOAD = "borexino_like toys: 2 datasets x 1200-bin domain, 16 species x 20000 fine points, gamma response, 23 params"

# Algorithmic FP32 floating-point operations per evaluated (bin, column) pair of
# the mixed generalized-gamma kernels on their branch-free path (shape d >= 50,
# 94% of the columns), FMA = 2, SFU reciprocal / exponential = 1:
#   forward  44 = offset and t (3) + ln(1+t)-t series (20) + centre exponent (3)
#                 + 3 Gauss-Legendre nodes and their weighted sum (14) + 2-dataset contraction (4)
#   backward 70 = dataset weight (3) + offset and t (3) + series (20) + ln(1+t) (1) + exponent (3)
#                 + nodes (15) + value / ln / offset-weighted sums (8) + mean / variance
#                 coefficients (11) + four accumulations (8)
FLOP_PER_PAIR = {"forward": 44, "backward": 70}
# The same count for the generalized gamma of free power p (--power), general per-node kernels, linear
# bins (3 nodes; the side nodes from the centre by the addition formula of e^q-1-q), |p L| <= 1/2:
#   forward   75 = offset and t (3) + ln(1+t) series (21) + centre L, pL, series and e1 (22)
#                  + side-node L and Q (8) + three exponents (9) + 3 exp2 (3) + weighted sum (5)
#                  + 2-dataset contraction (4)
#   backward 152 = offset, t and ln(1+t) (24) + centre (21) + side-node L, Q and e1 (16)
#                  + per node [exponent, exp2, weight and four node sums (13)] x 3 + dataset weight (3)
#                  + four compensated band sums (28) + three compensated rate sums (21)
FLOP_PER_PAIR_GG = {"forward": 75, "backward": 152}
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--toys", type=int, default=8192)
    ap.add_argument("--fp64-toys", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mv-toys", type=int, default=1024, help="toys of the multivariate workload")
    ap.add_argument("--fit-toys", type=int, default=1024, help="toys of the discovery-test workload")
    ap.add_argument("--minimiser", default="newton", choices=["newton", "lbfgs"],
                    help="discovery workload: batched Newton rate fits, or L-BFGS with window scales")
    ap.add_argument("--secondary", default=None, metavar="QxM",
                    help="toys workload with a secondary observable on both datasets: Q energy slices with "
                         "M secondary bins each (section 2.4 multivariate pieces), e.g. 8x16")
    ap.add_argument("--power", type=float, default=None,
                    help="toys workload with the generalized-gamma response of this free power p instead of "
                         "the gamma response (p is a 24th parameter, perturbed per toy like the others)")
    ap.add_argument("--workload", default="toys",
                    choices=["toys", "single", "species", "multivariate", "templates", "discovery"],
                    help="toys: the batched pseudo-experiments (default); single: sequential single-point "
                         "NLL + gradient calls; species: gsn_eval with a response-cache miss (tensor cores); "
                         "multivariate: batched toys of the 2-D workload (4 x 64 slices); templates: batched "
                         "toys of a Monte Carlo template fit (no response); discovery: batched profile-"
                         "likelihood fits (signal free and fixed at 0) of the toys")
    return ap.parse_args()


# ------------------------------------------------------------ inputs -------
def rank_toy_seed(rank, n_toys):
    """First toy seed of a rank's batch: ranks draw disjoint toys (weak scaling, no exchange)."""
    return 1000 + rank * n_toys


def max_over_ranks(value, dist, device):
    """The job's step time: the slowest rank's, returned to every rank (value itself on one rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, n_toys, ms):
    """Whole-job evaluations per second: every rank's toys over the slowest rank's step time."""
    return world * n_toys / (ms * 1e-3)


def make_inputs(n_toys, seed0, power=None, secondary=None):
    """Toys of the 1200-bin workload; with a power p, the generalized-gamma response (the counts are
    still drawn from the gamma response's expectation: only the model evaluated differs).  With a
    secondary observable ("QxM"), each toy also carries the secondary histograms, drawn from their
    expectation at theta0 (per-species slice sums of the FP64 GPU path's expected counts)."""
    import numpy as np

    from paper_1812_05686_gb300 import inputs as I
    w = I.borexino_like(n_bins=1200)
    if power is not None:
        w = I.with_power(w, power)
    mu0 = np.loadtxt(os.path.join(ROOT, "tests", "golden", "borexino_like_1200_mu0.txt"))
    ms = None
    if secondary is not None:
        from paper_1812_05686_gb300 import gsn
        Q, M = (int(v) for v in secondary.lower().split("x"))
        w = I.with_secondary(w, n_slices=Q, n_sec=M)
        ctx = gsn.context_from_workload(w, gsn.GSN_FP64)
        parts = []
        for d in range(2):
            per = ctx.expected(w["theta0"], d)
            x = w["secondary"][d]
            st, P = x["slice_start"], np.asarray(x["shapes"], np.float64)
            P = P / P.sum(axis=2, keepdims=True)
            N = np.stack([per[st[q]:st[q + 1]].sum(axis=0) for q in range(Q)], axis=1)
            parts.append(np.einsum("sq,sqm->qm", N, P).ravel())
        ms = np.concatenate(parts)
    b = I.toy_batch(w, [mu0[:1200], mu0[1200:]], n_toys=n_toys, seed0=seed0, mu_sec=ms)
    return w, b


# ------------------------------------------------------------ clocks -------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------ traffic ------
def ncu_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_mixed_gamma.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"kernel_sources_sha256:\s*([0-9a-f]+)", txt)
    t = re.search(r"traffic_bytes_per_launch_full:\s*([0-9.eE+]+)", txt)
    if not (m and t):
        return None
    return float(t.group(1)) if m.group(1) == kernel_sha() else None


KERNEL_SOURCES = ("gsn_mixed.cu", "gsn_device.cuh", "gsn_internal.cuh")


def kernel_sha():
    """Hash of the sources of the mixed-precision forward and adjoint kernels."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1812_05686_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------ gradient scale -----
def fisher_diagonal(ctx64, w, theta):
    """F_ii = sum_dj (d mu_dj / d theta_i)^2 / mu_dj at theta over the whole histograms.

    The statistical scale of each gradient component: sqrt(F_ii) is the spread of dNLL/dtheta_i
    from Poisson fluctuations of the counts.  Derivatives by central differences of the FP64
    GPU path's expected counts (gsn_expected), steps 1e-4 relative.
    """
    import numpy as np
    D = len(w["edges"])
    mu = [ctx64.expected(theta, d).sum(axis=1) for d in range(D)]
    F = np.zeros(len(theta))
    for i in range(len(theta)):
        h = 1e-4 * max(abs(theta[i]), 1e-6)
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        for d in range(D):
            dm = (ctx64.expected(tp, d).sum(axis=1) - ctx64.expected(tm, d).sum(axis=1)) / (2 * h)
            ok = mu[d] > 0
            F[i] += float(np.sum(dm[ok] ** 2 / mu[d][ok]))
    return F


def gradient_errors(gm, g64, F, names=None):
    """Mixed-vs-FP64 gradient errors per toy: normwise and per component on the Fisher scale."""
    import numpy as np
    norm = np.max(np.abs(gm - g64), axis=1) / np.maximum(np.max(np.abs(g64), axis=1), 1.0)
    comp = np.abs(gm - g64) / np.maximum(np.abs(g64) + np.sqrt(F)[None, :], 1.0)
    fish = np.max(comp, axis=1)
    worst = int(np.argmax(np.max(comp, axis=0)))
    return {"normwise_max": float(norm.max()), "normwise_median": float(np.median(norm)),
            "normwise_p99": float(np.percentile(norm, 99)), "toys_normwise_above_1e-5": int(np.sum(norm >= 1e-5)),
            "fisher_scaled_max": float(fish.max()), "fisher_scaled_median": float(np.median(fish)),
            "toys_fisher_scaled_above_1e-5": int(np.sum(fish >= 1e-5)),
            "fisher_scaled_worst_parameter": names[worst] if names else worst,
            "definition": "normwise: ||g - g64||_inf / max(||g64||_inf, 1); fisher_scaled: "
                          "max_i |g_i - g64_i| / max(|g64_i| + sqrt(F_ii), 1), F the Fisher diagonal at theta0 "
                          "over the whole histograms"}


# ------------------------------------------------------------- oracle ------
ORACLE_FINE = 2500     # fine columns of the oracle sample (the timed GPU workload has 20000)
ORACLE_SAMPLE = ("NLL + full gradient of one toy per process and step (toys of the batched workload: 2 datasets x "
                 "1200 bins, 16 species, each toy its own counts, window and parameters), FP64 oracle, on a "
                 "2500-point fine grid (the GPU workload has 20000 points)")
ORACLE_FULL_GRID = ("x 2500/20000: the oracle's cost is linear in the fine columns (every (bin, column) pair is "
                    "evaluated); an estimate, not a measurement")
_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
_ORACLE = {}


def _oracle_setup():
    import numpy as np

    from oracle import gsn_oracle as O
    from paper_1812_05686_gb300 import inputs as I
    if not _ORACLE:
        w = I.borexino_like(n_bins=1200, n_fine=ORACLE_FINE)
        mu0 = np.loadtxt(os.path.join(ROOT, "tests", "golden", "borexino_like_1200_mu0.txt"))
        _ORACLE.update(O=O, I=I, w=w, mu=[mu0[:1200], mu0[1200:]])
    return _ORACLE


def _oracle_warm(_):
    """Pool job: import the oracle and build the sample workload (untimed); the pause lets every
    process of the pool take one of these jobs."""
    _oracle_setup()
    time.sleep(1.0)
    return os.getpid()


def _oracle_toy(t):
    """Pool job: the oracle's NLL and gradient of toy t of the sample workload; returns seconds."""
    o = _oracle_setup()
    b = o["I"].toy_batch(o["w"], o["mu"], n_toys=1, seed0=1000 + t)
    t0 = time.perf_counter()
    o["O"].nll(o["w"], b["params"][0], b["counts"][0], b["windows"][0])
    o["O"].nll_grad(o["w"], b["params"][0], b["counts"][0], b["windows"][0])
    return time.perf_counter() - t0


def oracle_steps(n_steps, procs):
    """Wall seconds of n_steps oracle steps; a step is one toy on each of `procs` processes at once
    (spawn pool, one BLAS thread per process)."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    os.environ.update({k: "1" for k in _THREAD_VARS})
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            pool.map(_oracle_warm, range(procs), chunksize=1)
            out = []
            for s in range(n_steps):
                t0 = time.perf_counter()
                pool.map(_oracle_toy, [s * procs + i for i in range(procs)], chunksize=1)
                out.append(time.perf_counter() - t0)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return out


def host_cores():
    return len(os.sched_getaffinity(0))


def cpu_baseline_record():
    """The oracle on this host: one process per core over toys (the baseline value) and one process
    alone, both measured on the 2500-point sample; the full-grid figure is a separate estimate."""
    cores = host_cores()
    single = oracle_steps(1, 1)[0]
    allc = oracle_steps(1, cores)[0]
    return {"value": cores / allc, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": ORACLE_SAMPLE + f"; {cores} processes, one toy each, timed together",
            "fine_points": ORACLE_FINE,
            "single_thread": {"value": 1.0 / single, "unit": UNIT, "cores": 1, "seconds_per_toy": single},
            "full_grid_estimate": {"value": cores / allc * ORACLE_FINE / 20000, "unit": UNIT, "basis": ORACLE_FULL_GRID}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cores = host_cores()
    ts = oracle_steps(args.warmup + args.steps, cores)[args.warmup:]
    sec = sum(ts) / len(ts)
    value = cores / sec
    sample = ORACLE_SAMPLE + f"; {cores} processes, one toy each per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("20000 fine points", f"{ORACLE_FINE} fine points"),
                       "toys_per_step": cores, "fine_points": ORACLE_FINE, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "full_grid_estimate": {"value": value * ORACLE_FINE / 20000, "unit": UNIT, "basis": ORACLE_FULL_GRID},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- ours ------
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1812_05686_gb300 import gsn

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    T = args.toys
    w, b = make_inputs(T, rank_toy_seed(rank, T), args.power, args.secondary)
    gg = args.power is not None
    sec = args.secondary is not None
    # a dedicated stream: the library launches on it and the timing events are recorded on it
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = gsn.context_from_workload(w, gsn.GSN_MIXED, device=local_rank, stream=stream.cuda_stream)
    P, B, D = w["n_params"], b["counts"].shape[1], 2
    params = torch.from_numpy(b["params"]).to(dev)
    counts = torch.from_numpy(b["counts"]).to(dev)
    wins = torch.from_numpy(b["windows"].astype(np.int32)).to(dev)
    nll = torch.empty(T, dtype=torch.float64, device=dev)
    grad = torch.empty(T, P, dtype=torch.float64, device=dev)
    status = torch.empty(T, dtype=torch.int32, device=dev)

    def step():
        rc = ctx.eval_grad_batch_dev(params, counts, wins, nll, grad, status)
        if rc != 0:
            raise RuntimeError(ctx.last_error())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ctx.profile(True)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    prof = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist, dev)
    st = status.cpu().numpy()
    nll_mixed = nll.cpu().numpy()
    value = job_rate(world, T, ms)

    # FP64 path on a stride of toys over the whole batch (every launch chunk): throughput and the
    # mixed path's errors against it (--fp64-toys 0: skipped)
    nf = min(args.fp64_toys, T)
    fp64 = None
    if nf > 0:
        idx = (np.arange(nf) * T) // nf
        sel = torch.from_numpy(idx).to(dev)
        p_s, c_s, w_s = params[sel].contiguous(), counts[sel].contiguous(), wins[sel].contiguous()
        ctx64 = gsn.context_from_workload(w, gsn.GSN_FP64, device=local_rank, stream=stream.cuda_stream)
        nll64 = torch.empty(nf, dtype=torch.float64, device=dev)
        grad64 = torch.empty(nf, P, dtype=torch.float64, device=dev)
        torch.cuda.synchronize(dev)
        ctx64.eval_grad_batch_dev(p_s, c_s, w_s, nll64, grad64, None)
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        ctx64.eval_grad_batch_dev(p_s, c_s, w_s, nll64, grad64, None)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        fp64_value = nf / (f0.elapsed_time(f1) * 1e-3)
        dnll = float(np.max(np.abs(nll64.cpu().numpy() - nll_mixed[idx])))
        gerrs = gradient_errors(grad.cpu().numpy()[idx], grad64.cpu().numpy(), fisher_diagonal(ctx64, w, w["theta0"]),
                               w.get("param_names"))
        chunk = 4096
        fp64 = {"value": fp64_value, "unit": UNIT, "toys": nf,
                "toy_sample": f"every {T // nf}th toy of the {T} (toys {int(idx[0])}..{int(idx[-1])}; launch chunks "
                              f"of {chunk}: {sorted(set(int(i) // chunk for i in idx))})",
                "speedup_mixed_over_fp64": value / world / fp64_value,
                "max_abs_dnll_mixed_vs_fp64": dnll, "grad_normwise_err_mixed_vs_fp64": gerrs["normwise_max"],
                "grad_err_mixed_vs_fp64": gerrs}

    # the same step replayed from a CUDA graph (tracing off: no events between the kernels)
    for _ in range(2):
        step()
    torch.cuda.synchronize(dev)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        step()
    g1.record(stream)
    torch.cuda.synchronize(dev)
    graph_ms = g0.elapsed_time(g1) / args.steps

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        hp, hc, hw = b["params"], b["counts"], b["windows"].astype(np.int32)
        ctx.eval_grad_batch(hp, hc, hw)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(max(1, min(args.steps, 3))):
            rc, _, _ = ctx.eval_grad_batch(hp, hc, hw)
        dt = (time.perf_counter() - t0) / max(1, min(args.steps, 3))
        h2d = T * (P * 8 + B * 8 + D * 2 * 4)
        d2h = T * (8 + P * 8 + 4)
        e2e = {"value": world * T / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # roofline of the dominant kernel (event time per launch, algorithmic FLOPs per launch)
    dom = max(("forward", "backward"), key=lambda k: prof[k][0])
    kms, kn, kunits = prof[dom]
    per_launch_s = kms * 1e-3 / max(kn, 1)
    flops = kunits / max(kn, 1) * (FLOP_PER_PAIR_GG if gg else FLOP_PER_PAIR)[dom] if kunits else 0.0
    sm_mhz = clk.get("sm_mhz") or 1455.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = nsm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6
    achieved = flops / per_launch_s
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None if (gg or sec) else ncu_traffic(dom), "kernel": dom,
            "peak_basis": f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x median SM clock {sm_mhz:.0f} MHz",
            "pairs_per_launch": kunits / max(kn, 1), "ms_per_launch": per_launch_s * 1e3}
    # method-level figures beside the FLOP fraction: (bin, column) pairs per second of both response
    # kernels against the measured rate of one quadrature node (2 FFMA + EX2 + FFMA, three nodes per
    # pair), and the FLOP rate against the measured FFMA rate (probes outside the timed region)
    node_rate = gsn.peak_probe(gsn.GSN_PROBE_NODE, local_rank)
    ffma_rate = gsn.peak_probe(gsn.GSN_PROBE_FFMA, local_rank)
    roof["frac_of_measured_ffma"] = achieved / (2.0 * ffma_rate)
    roof["measured_ffma_tflops"] = 2.0 * ffma_rate / 1e12
    method = {}
    for kname in ("forward", "backward"):
        kms_, kn_, ku_ = prof[kname]
        if kn_ and ku_:
            pps = ku_ / (kms_ * 1e-3)
            method[kname] = {"pairs_per_s": pps, "node_evals_per_s": 3.0 * pps, "measured_node_peak_per_s": node_rate,
                             "frac_of_node_peak": 3.0 * pps / node_rate}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_record()

    # the gamma forward's launcher also runs its one-block segment prefix (not a traced kernel class)
    launches = sum(v[1] for v in prof.values()) + (0 if gg else prof["forward"][1])
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32 (f64 deviance and reductions)", "data": "synthetic",
                "config": {"workload": (WORKLOAD if not gg else
                           WORKLOAD.replace("gamma response, 23 params",
                                            f"generalized-gamma response of free power p = {args.power:g}, 24 params"))
                           + (f"; secondary observable {args.secondary} (slices x bins) per dataset" if sec else ""),
                           "toys_per_gpu": T, "fine_points": 20000, "bins": 1200,
                           "species": 16, "precision": "mixed",
                           "l2": "inputs and scratch per step (GBs) exceed the 129 MB L2"},
                "fp64_path": fp64,
                "graph_replay": {"value": world * T / (graph_ms * 1e-3), "unit": UNIT, "ms_per_step": graph_ms,
                                 "note": "same step replayed from one CUDA graph with tracing off; the headline "
                                         "value is the traced run (events around every launch)"},
                "plan": ctx.plan_info(min(T, 4096), True),
                "status_nonzero_toys": int(np.count_nonzero(st)),
                "roofline": roof, "pairs_vs_node_peak": method, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches,
                "kernels": {k: {"ms_total": v[0], "launches": v[1], "pairs": v[2]} for k, v in prof.items() if v[1]}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_single(args):
    """Sequential single-point gsn_eval_grad calls (a minimiser's loop): host buffers, one call per step."""
    import numpy as np
    import torch

    from paper_1812_05686_gb300 import gsn, inputs as I
    torch.cuda.init()
    out = []
    for name, work, mu_file in (("single_gauss 900 bins x 2000 fine points, 8 species", I.single_gauss(), None),
                                ("borexino_like 2 x 1000 bins x 20000 fine points, 16 species", I.borexino_like(), None)):
        rng = np.random.Generator(np.random.PCG64(9))
        counts = [rng.poisson(50.0, len(e) - 1).astype(np.float64) for e in work["edges"]]
        pts = I.perturbed_points(work["theta0"], 64, 2)
        for prec, label in ((gsn.GSN_MIXED, "mixed"), (gsn.GSN_FP64, "fp64")):
            n = 64 if prec == gsn.GSN_MIXED else 16
            rec = {"workload": name, "precision": label, "calls": n}
            for graphs in (1, 0):
                ctx = gsn.context_from_workload(work, prec, counts=counts, use_graphs=graphs)
                for p in pts[:4]:
                    ctx.eval_grad(p)
                t0 = time.perf_counter()
                for i in range(n):
                    rc, v, g = ctx.eval_grad(pts[i % len(pts)])
                dt = (time.perf_counter() - t0) / n
                if graphs:
                    rec.update({"ms_per_call": dt * 1e3, "evals_per_s": 1.0 / dt, "plan": ctx.plan_info(1, True)})
                    # per-kernel event times of the same calls (tracing on: plain launches)
                    ctx.profile(True)
                    for i in range(n):
                        ctx.eval_grad(pts[i % len(pts)])
                    prof = ctx.profile_read()
                    ctx.profile(False)
                    rec["kernel_us_per_call"] = {k: 1e3 * v[0] / n for k, v in prof.items() if v[1]}
                else:
                    rec["ms_per_call_without_graphs"] = dt * 1e3
                ctx.close()
            out.append(rec)
    print(json.dumps({"metric": "sequential NLL+grad calls (gsn_eval_grad, host buffers)", "unit": "evals/s",
                      "data": "synthetic", "results": out}), flush=True)


def run_species(args):
    """gsn_eval with a response-cache miss on every call: the tcgen05 per-species contraction."""
    import numpy as np
    import torch

    from paper_1812_05686_gb300 import gsn, inputs as I
    torch.cuda.init()
    work = I.borexino_like()
    rng = np.random.Generator(np.random.PCG64(9))
    counts = [rng.poisson(50.0, len(e) - 1).astype(np.float64) for e in work["edges"]]
    ctx = gsn.context_from_workload(work, gsn.GSN_MIXED, counts=counts)
    p = work["theta0"].copy()
    LY = work["param_names"].index("LY")
    for i in range(3):
        p[LY] = 500.0 + 1e-3 * i
        ctx.eval(p)
    ctx.profile(True)
    n = 50
    t0 = time.perf_counter()
    for i in range(n):
        p[LY] = 500.0 + 1e-3 * (i + 10)   # a new light yield: the cached per-species shapes are recomputed
        rc, v = ctx.eval(p)
    dt = (time.perf_counter() - t0) / n
    prof = ctx.profile_read()
    ctx.profile(False)
    ms, launches, pairs = prof["species"]
    S_pad = 16
    tc_flop = 3 * 2 * S_pad * (pairs / max(launches, 1))       # split-TF32: three products per pair
    useful = 2 * work["spectra"].shape[0] * (pairs / max(launches, 1))
    per_launch = ms * 1e-3 / max(launches, 1)
    peak_tf32 = 1925.7e12 / 2  # measured bf16 dense peak x the nominal tf32 / bf16 ratio
    print(json.dumps({"metric": "gsn_eval with response recomputation (per-species contraction on tensor cores)",
                      "value": 1.0 / dt, "unit": "evals/s", "precision": "mixed", "data": "synthetic",
                      "config": {"workload": "borexino_like 2 x 1000 bins x 20000 fine points, 16 species"},
                      "species_kernel": {"ms_per_launch": per_launch * 1e3, "pairs_per_launch": pairs / max(launches, 1),
                                         "tensor_tflops_issued": tc_flop / per_launch / 1e12,
                                         "useful_tflops": useful / per_launch / 1e12,
                                         "tf32_peak_tflops": peak_tf32 / 1e12,
                                         "tensor_frac": tc_flop / per_launch / peak_tf32},
                      "kernels": {k: {"ms_total": v[0], "launches": v[1]} for k, v in prof.items() if v[1]}}),
          flush=True)


MV_WORKLOAD = ("multivariate_like: 4 datasets x 64 slices (energy x second observable) x 1000 bins, 32 species x "
               "50000 fine points, gamma response, per-slice LY and a multipliers and rate fractions, 37 params")


def run_multivariate(args):
    """Batched toys of the 2-D multivariate workload, mixed path timed, FP64 path on the first toys."""
    import numpy as np
    import torch

    from paper_1812_05686_gb300 import gsn, inputs as I
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    w = I.multivariate_like()
    D, P, T = len(w["edges"]), w["n_params"], args.mv_toys
    nb = len(w["edges"][0]) - 1
    ctx = gsn.context_from_workload(w, gsn.GSN_MIXED, stream=stream.cuda_stream)
    # benchmark input only: the Asimov mean at theta0 from the mixed path (one response evaluation)
    mu0 = np.concatenate([ctx.expected(w["theta0"], d).sum(axis=1) for d in range(D)])
    gen = torch.Generator(device=dev)
    gen.manual_seed(1000)
    counts = torch.poisson(torch.from_numpy(mu0).to(dev).expand(T, -1).contiguous(), generator=gen)
    params = torch.from_numpy(I.perturbed_points(w["theta0"], T, 1000 + T)).to(dev)
    wins = torch.zeros(T, D, 2, dtype=torch.int32, device=dev)
    wins[:, :, 1] = nb
    nll = torch.empty(T, dtype=torch.float64, device=dev)
    grad = torch.empty(T, P, dtype=torch.float64, device=dev)
    status = torch.empty(T, dtype=torch.int32, device=dev)

    def step():
        rc = ctx.eval_grad_batch_dev(params, counts, wins, nll, grad, status)
        if rc != 0:
            raise RuntimeError(ctx.last_error())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    ctx.profile(True)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    prof = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    value = T / (ms * 1e-3)
    fp64 = None
    nf = min(args.fp64_toys, T, 4)
    if nf > 0:
        ctx64 = gsn.context_from_workload(w, gsn.GSN_FP64, stream=stream.cuda_stream)
        n64 = torch.empty(nf, dtype=torch.float64, device=dev)
        g64 = torch.empty(nf, P, dtype=torch.float64, device=dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        rc = ctx64.eval_grad_batch_dev(params[:nf], counts[:nf], wins[:nf], n64, g64, None)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        if rc != 0:
            raise RuntimeError(ctx64.last_error())
        gm, gd = grad[:nf].cpu().numpy(), g64.cpu().numpy()
        norm = np.max(np.abs(gm - gd), axis=1) / np.maximum(np.max(np.abs(gd), axis=1), 1.0)
        fp64 = {"value": nf / (f0.elapsed_time(f1) * 1e-3), "unit": UNIT, "toys": nf,
                "max_abs_dnll_mixed_vs_fp64": float(np.max(np.abs(n64.cpu().numpy() - nll[:nf].cpu().numpy()))),
                "grad_normwise_err_mixed_vs_fp64": float(norm.max())}
    dom = max(("forward", "backward"), key=lambda k: prof[k][0])
    kms, kn, kunits = prof[dom]
    per_launch_s = kms * 1e-3 / max(kn, 1)
    sm_mhz = clk.get("sm_mhz") or 1455.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = nsm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6
    achieved = kunits / max(kn, 1) * FLOP_PER_PAIR[dom] / per_launch_s
    line = {"metric": "NLL+grad evals/sec (batched toys, 2-D multivariate workload) on 1 GB300", "value": value,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "dtype": "f32 (f64 deviance and reductions)", "data": "synthetic",
            "config": {"workload": MV_WORKLOAD, "toys": T, "datasets": D, "precision": "mixed",
                       "plan": ctx.plan_info(min(T, 83), True)},
            "fp64_path": fp64, "status_nonzero_toys": int(torch.count_nonzero(status).item()),
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                         "frac": achieved / peak, "kernel": dom, "pairs_per_launch": kunits / max(kn, 1),
                         "ms_per_launch": per_launch_s * 1e3},
            "clocks": clk, "gpu_launches": sum(v[1] for v in prof.values()),
            "kernels": {k: {"ms_total": v[0], "launches": v[1], "pairs": v[2]} for k, v in prof.items() if v[1]}}
    print(json.dumps(line), flush=True)


TPL_WORKLOAD = ("template_like: Monte Carlo template fit, 2 datasets x 1000 bins, 16 template species "
                "(visible-bin histograms), 16 rate params, ragged windows 600-1000 bins")


def run_templates(args):
    """Batched toys of a pure template fit: only the FP64 deviance stage runs (no response)."""
    import numpy as np
    import torch

    from paper_1812_05686_gb300 import gsn, inputs as I
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    w = I.template_like()
    D, P, T = len(w["edges"]), w["n_params"], args.toys
    nb = len(w["edges"][0]) - 1
    ctx = gsn.context_from_workload(w, gsn.GSN_MIXED, stream=stream.cuda_stream)
    # benchmark input: the expected counts at theta0 from the library (templates times rates)
    mu0 = np.concatenate([ctx.expected(w["theta0"], d).sum(axis=1) for d in range(D)])
    gen = torch.Generator(device=dev)
    gen.manual_seed(2000)
    counts = torch.poisson(torch.from_numpy(mu0).to(dev).expand(T, -1).contiguous(), generator=gen)
    params = torch.from_numpy(I.perturbed_points(w["theta0"], T, 2000 + T)).to(dev)
    win = I.toy_windows(T, nb, 600, 1000, 2000 + 2 * T)
    wins = torch.from_numpy(np.repeat(win[:, None, :], D, axis=1).astype(np.int32)).to(dev)
    nll = torch.empty(T, dtype=torch.float64, device=dev)
    grad = torch.empty(T, P, dtype=torch.float64, device=dev)
    status = torch.empty(T, dtype=torch.int32, device=dev)

    def step():
        rc = ctx.eval_grad_batch_dev(params, counts, wins, nll, grad, status)
        if rc != 0:
            raise RuntimeError(ctx.last_error())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    ctx.profile(True)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    prof = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    # roofline of the deviance stage: FP64, 2 FMA per template and bin (mu and the rate gradient)
    S = w["spectra"].shape[0]
    kms, kn, _ = prof["deviance"]
    per_launch_s = kms * 1e-3 / max(kn, 1)
    bins_per_launch = min(T, 4096) * D * nb
    flops = bins_per_launch * 4.0 * S
    dfma = gsn.peak_probe(gsn.GSN_PROBE_DFMA)
    hbm = bins_per_launch * (8 + 4)  # counts read, w written (FP32)
    line = {"metric": "NLL+grad evals/sec (batched toys, Monte Carlo template fit) on 1 GB300", "value": T / (ms * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "dtype": "f64 (template contraction and deviance)", "data": "synthetic",
            "config": {"workload": TPL_WORKLOAD, "toys": T},
            "status_nonzero_toys": int(torch.count_nonzero(status).item()),
            "roofline": {"bound": "alu (fp64)", "achieved": flops / per_launch_s / 1e12, "peak": 2 * dfma / 1e12,
                         "unit": "TFLOP/s", "frac": flops / per_launch_s / (2 * dfma), "kernel": "deviance",
                         "peak_basis": "measured DFMA rate (gsn_peak_probe) x 2",
                         "hbm_gbs": hbm / per_launch_s / 1e9, "ms_per_launch": per_launch_s * 1e3},
            "clocks": clk, "gpu_launches": sum(v[1] for v in prof.values()),
            "kernels": {k: {"ms_total": v[0], "launches": v[1]} for k, v in prof.items() if v[1]}}
    print(json.dumps(line), flush=True)


def run_discovery(args):
    """Toy Monte Carlo discovery test on the batched pseudo-experiment workload: every toy in its own
    window (600..1200 bins), two batched L-BFGS fits per toy with all 16 rates free (>= 0), the
    second with the signal rate fixed at 0; q0 = 2 (NLL_fixed - NLL_free).  Per-toy scales: the
    rates' 1/sqrt(Fisher) over the whole histograms at theta0, widened per toy by
    gsn_window_scales_dev for the part of each species outside the toy's window."""
    import numpy as np
    import torch

    from paper_1812_05686_gb300 import gsn
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    T = args.fit_toys
    w, b = make_inputs(T, 1000)
    P, D, S = w["n_params"], 2, w["spectra"].shape[0]
    ctx = gsn.context_from_workload(w, gsn.GSN_MIXED, stream=stream.cuda_stream)
    tot = sum(ctx.expected(w["theta0"], d).sum(axis=0) for d in range(D))
    rates = np.unique(w["slot_map"][:, :S][w["slot_map"][:, :S] >= 0])
    free = np.zeros(P, bool)
    free[rates] = True
    # scales 1 / sqrt(Fisher diagonal) of the rates at theta0 over the whole histograms (d mu / d r_s = mu_s / r_s)
    fis = np.zeros(P)
    for d in range(D):
        per = ctx.expected(w["theta0"], d)
        m = per.sum(axis=1)
        ok = m > 0
        for s in range(S):
            p = w["slot_map"][d, s]
            if p >= 0 and w["theta0"][p] > 0:
                fis[p] += float(np.sum((per[ok, s] / w["theta0"][p]) ** 2 / m[ok]))
    scale = np.where(free & (fis > 0), 1.0 / np.sqrt(np.where(fis > 0, fis, 1.0)), 1.0)
    lo = np.where(free, 0.0, -np.inf)
    # the species with the fewest counts among those with more than 2% of the largest plays the signal
    fitted = [s for s in range(S) if tot[s] > 0.02 * tot.max()]
    sig = int(w["slot_map"][0, min(fitted, key=lambda s: tot[s])])
    counts = torch.from_numpy(b["counts"]).to(dev)
    wins = torch.from_numpy(b["windows"].astype(np.int32)).to(dev)
    start = np.repeat(w["theta0"][None, :], T, axis=0)
    start0 = start.copy()
    start0[:, sig] = 0.0
    free0 = free.copy()
    free0[sig] = False
    torch.cuda.synchronize(dev)
    EDM = 1e-5  # stop at an estimated distance to the minimum of 1e-5 in NLL (q0 to 2e-5)

    newton = args.minimiser == "newton"

    def fits():
        x1 = torch.from_numpy(start.copy()).to(dev)
        x0 = torch.from_numpy(start0.copy()).to(dev)
        if newton:  # exact Newton on the rates (the response held): gsn_fit_rates_batch_dev
            f1, e1, s1 = ctx.fit_rates_batch_dev(x1, counts, wins, free=free, lo=lo)
            f0, e0, s0 = ctx.fit_rates_batch_dev(x0, counts, wins, free=free0, lo=lo)
        else:       # L-BFGS with per-toy window scales and the EDM rule
            sc1 = ctx.window_scales_dev(x1, wins, scale=scale)
            f1, e1, s1 = ctx.minimize_batch_dev(x1, counts, wins, free=free, lo=lo, max_evals=300, scale_dev=sc1,
                                                edm=EDM)
            f0, e0, s0 = ctx.minimize_batch_dev(x0, counts, wins, free=free0, lo=lo, max_evals=300, scale_dev=sc1,
                                                edm=EDM)
        return f1, e1, s1, f0, e0, s0

    fits()  # warm-up: plans, graphs
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    f1, e1, s1, f0, e0, s0 = fits()
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    clk = clocks.stop()
    q0 = np.maximum(0.0, 2.0 * (f0.cpu().numpy() - f1.cpu().numpy()))
    ev = np.concatenate([e1.cpu().numpy(), e0.cpu().numpy()])
    st = np.concatenate([s1.cpu().numpy(), s0.cpu().numpy()])
    line = {"metric": "profile-likelihood fits/sec (batched toys, discovery test) on 1 GB300", "value": 2 * T / dt,
            "unit": "fits/s", "n_gpus": 1, "ms_total": dt * 1e3, "higher_is_better": True,
            "dtype": "f32 response, f64 deviance and minimiser state", "data": "synthetic",
            "config": {"workload": WORKLOAD + "; every toy in its own window (600..1200 bins)", "toys": T,
                       "free": [w["param_names"][i] for i in np.nonzero(free)[0]], "signal": w["param_names"][sig],
                       "minimiser": ("projected Newton on the rates with the exact Hessian (response held), "
                                     "stop at a Newton decrement / 2 below 1e-8") if newton else
                                    ("projected L-BFGS per toy, history 16, per-toy window scales, stop at "
                                     "gtol 1e-4 (scaled) or an estimated distance to the minimum below 1e-5")},
            ("newton_iterations_per_fit" if newton else "evals_per_fit"): {"mean": float(ev.mean()), "max": int(ev.max())},
            "status_counts": {str(k): int(v) for k, v in zip(*np.unique(st, return_counts=True))},
            "q0": {"median": float(np.median(q0)), "p90": float(np.percentile(q0, 90)), "max": float(q0.max())},
            **({} if newton else {"nll_evals_per_s": float(ev.sum() * 1.0 / dt)}), "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "single":
        return run_single(args)
    if args.workload == "species":
        return run_species(args)
    if args.workload == "multivariate":
        return run_multivariate(args)
    if args.workload == "templates":
        return run_templates(args)
    if args.workload == "discovery":
        return run_discovery(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
