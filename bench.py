"""Benchmark of the TSM loop path on GB300 (one JSON line on rank 0).

Workload (N = 1): 24^3 x 48 lattice, near-unit SU(3) links exp(0.25 i H)
(seed 3), kappa = 0.1245, mu = 0.005, antiperiodic t, Z4 noise; N_HP = 8 HP
solves (FP32 iterations with FP64 reliable updates, rel. residual 1e-10) and
N_LP = 256 LP solves (FP16 storage, FP32 arithmetic, truncated at 5e-3 or 60
iterations); loops for 16 insertions at 7 momenta; TSM combine.  One step =
one complete TSM estimate (264 sources) with fresh noise (seed per step).

metric: TSM sources/s.  Alongside: the equal-loop-error comparison with the
plain FP64 path (every source solved to 1e-10 in FP64, standard estimator),
the hop-kernel roofline (CUDA events on the library's stream inside the timed
region), standalone Dslash GB/s per tier, the end-to-end number through the C
ABI with host buffers, the oracle's CPU throughput on a bounded sample, the
clocks seen during the timed region and the kernel-launch count.

--impl reference runs the CPU oracle (the only other implementation of this
method here) on the same workload, on every host core at once (one spawned
worker process per core): a warm-up step runs one complete LP source per
worker (LP iteration count and per-source time), each further step one
application of the Schur operator at 24^3 x 48 per worker; scaled to
sources/s and summed over the cores.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (24, 24, 24, 48)
EPS, KAPPA, MU, GAUGE_SEED = 0.25, 0.1245, 0.005, 3
N_HP, N_LP = 8, 256
HP_TOL, LP_TOL, LP_MAXIT, HP_MAXIT = 1e-10, 5e-3, 60, 20000
RELIABLE_DELTA = 1e-5        # FP64 residual replacement whenever ||r|| fell by 10^5
TIERS = {0: "f64", 1: "f32", 2: "bf16", 3: "f16"}
REAL_BYTES = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}
NAIVE_REALS = {"f64": 8 * 18 + 8 * 24 + 24, "f32": 312, "bf16": 312, "f16": 312}
KINDS = ("K1_hop", "K2_hop_xpay_norm", "K3_hop_dag", "K4_hop_dag_cg_update")
N_GAMMA, N_Q = 16, 7
METRIC = "TSM sources/sec at 24^3x48 and Dslash HBM GB/s, vs plain FP64 at equal loop error"
WORKLOAD = "tsm-24^3x48-eps0.25-k0.1245-mu0.005-Z4-hp8(f32+f64rel,1e-10)-lp256(f16,5e-3|60)-16G-7q"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip e2e / equal-error / cpu-baseline legs")
    ap.add_argument("--batch", type=int, default=None,
                    help="sources solved together (multi-RHS kernels); default: the autotuner's choice (tsm_tune: "
                         "batch width and sources per link-sharing block of the FP16 stencil)")
    ap.add_argument("--reliable-delta", type=float, default=None, help="override the HP reliable-update delta")
    ap.add_argument("--hp-warm-start", action="store_true",
                    help="HP solves start from their source's LP solution instead of zero")
    ap.add_argument("--mode", default="eager", choices=["eager", "graph"],
                    help="eager: host-driven chunked CG loops; graph: one captured CUDA graph per step "
                         "(device-side loops, LP set beside the HP set)")
    ap.add_argument("--workload", default="tsm24",
                    choices=["tsm24", "three-lattice", "learned", "scale", "estimators"],
                    help="tsm24: the headline 24^3x48 TSM step; three-lattice: 8^3x16 + 12^3x24 + 16^3x32 "
                         "in one captured graph (batching workload, its own JSON line); learned: the learned "
                         "LP preconditioner at 16^3x32 (training + held-out evaluation, its own JSON line); "
                         "scale: the full TSM at 32^3x64 with local and one-derivative insertions (its own "
                         "JSON line); estimators: the 24^3x48 step with each estimator (standard, one-end, "
                         "generalised one-end, derivative insertions, all momenta by FFT) and its kernels")
    ap.add_argument("--train-steps", type=int, default=400, help="learned workload: Adam steps")
    ap.add_argument("--pairs-per-field", type=int, default=500, help="learned workload: pairs per training field")

    ap.add_argument("--net-only", action="store_true",
                    help="only run 3 forward passes of the learned preconditioner's network (channels "
                         "1-12-12-12-1) at 16^3x32, timed with CUDA events (a small case for ncu captures of "
                         "the transport and tensor-core GEMM kernels)")
    ap.add_argument("--lp-only", action="store_true",
                    help="only run one batched LP solve (32 Z4 sources, FP16 storage, 5e-3 or 60 iterations) at "
                         "16^3x32 (a small case for ncu captures of the batched K1-K4 kernels; its fields exceed "
                         "L2)")
    ap.add_argument("--fft-only", action="store_true",
                    help="only run two all-momenta TSM estimates of 64 LP sources (FP16, batch 32) at 24^3x48 (a "
                         "small case for ncu captures of the FFT projection kernels)")
    ap.add_argument("--contract-only", action="store_true",
                    help="only run one LP-only TSM estimate of 4 sources (FP16 solves, batch 4) at 24^3x48 with "
                         "16 Gamma x 7 momenta (a small case for ncu captures of the contraction kernel)")
    ap.add_argument("--dslash-only", default=None,
                    help="comma list of tiers (f64,f32,f16,bf16): only run 3 standalone H_eo launches per tier "
                         "at 24^3x48 (a small case for ncu captures of the hop kernel)")
    return ap.parse_args()


def run_net_only():
    import torch
    from paper_1211_0126_gb300 import build, tsm
    from paper_1211_0126_gb300 import synthetic as S
    if not os.path.exists(tsm.LIB_PATH):
        build.build()
    dims = (16, 16, 16, 32)
    V = int(np.prod(dims))
    stream = torch.cuda.current_stream()
    ctx = tsm.Context(0, stream.cuda_stream)
    ctx.load_gauge(S.gauge_field(dims, EPS, 201), dims, KAPPA, MU)
    net = tsm.Network([1, 12, 12, 12, 1], seed=7, init_scale=0.1)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(1, 1, V * 12, dtype=torch.complex128, device="cuda", generator=g)
    y = torch.zeros_like(x)
    tsm.tsm_net_forward(net.h, ctx.h, 1, x, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        tsm.tsm_net_forward(net.h, ctx.h, 1, x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    print(json.dumps({"net_only": {"lattice": list(dims), "channels": [1, 12, 12, 12, 1],
                                   "ms_per_forward": e0.elapsed_time(e1) / 3}}), flush=True)
    net.close()
    ctx.close()


def run_lp_only():
    import torch
    from paper_1211_0126_gb300 import build, tsm
    from paper_1211_0126_gb300 import synthetic as S
    if not os.path.exists(tsm.LIB_PATH):
        build.build()
    dims = (16, 16, 16, 32)
    stream = torch.cuda.current_stream()
    ctx = tsm.Context(0, stream.cuda_stream)
    ctx.load_gauge(S.gauge_field(dims, EPS, GAUGE_SEED), dims, KAPPA, MU)
    V = int(np.prod(dims))
    b = torch.zeros(32, V * 12, dtype=torch.complex128, device="cuda")
    for j in range(32):
        tsm.tsm_noise(ctx.h, 77, 4, j, b[j])
    s = torch.zeros_like(b)
    lp = tsm.stop(LP_TOL, LP_MAXIT, tsm.TSM_F16)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, iters, _ = tsm.tm_solve_batch(ctx.h, b, s, lp, 32)
    torch.cuda.synchronize()
    print(json.dumps({"lp_only": {"lattice": list(dims), "batch": 32, "iters_mean": float(np.mean(iters)),
                                  "ms": (time.perf_counter() - t0) * 1e3}}), flush=True)
    ctx.close()


def run_contract_only():
    import torch
    from paper_1211_0126_gb300 import build, tsm
    from paper_1211_0126_gb300 import synthetic as S
    if not os.path.exists(tsm.LIB_PATH):
        build.build()
    ctx = tsm.Context(0, torch.cuda.current_stream().cuda_stream)
    ctx.load_gauge(S.gauge_field(DIMS, EPS, GAUGE_SEED), DIMS, KAPPA, MU)
    hp = tsm.stop(HP_TOL, HP_MAXIT, tsm.TSM_F32, reliable=True, reliable_delta=RELIABLE_DELTA)
    lp = tsm.stop(LP_TOL, LP_MAXIT, tsm.TSM_F16)
    t0 = time.perf_counter()
    ctx.loops(5, 4, 0, 4, hp, lp, list(range(N_GAMMA)), S.default_momenta(N_Q), batch=4, verify=False)
    torch.cuda.synchronize()
    print(json.dumps({"contract_only": {"lattice": list(DIMS), "lp_sources": 4, "n_gamma": N_GAMMA, "n_q": N_Q,
                                        "ms": (time.perf_counter() - t0) * 1e3}}), flush=True)
    ctx.close()


def run_fft_only():
    import torch
    from paper_1211_0126_gb300 import build, tsm
    from paper_1211_0126_gb300 import synthetic as S
    if not os.path.exists(tsm.LIB_PATH):
        build.build()
    ctx = tsm.Context(0, torch.cuda.current_stream().cuda_stream)
    ctx.load_gauge(S.gauge_field(DIMS, EPS, GAUGE_SEED), DIMS, KAPPA, MU)
    hp = tsm.stop(HP_TOL, HP_MAXIT, tsm.TSM_F32, reliable=True, reliable_delta=RELIABLE_DELTA)
    lp = tsm.stop(LP_TOL, LP_MAXIT, tsm.TSM_F16)
    t0 = time.perf_counter()
    for k in range(2):
        ctx.loops(5 + k, 4, 0, 64, hp, lp, list(range(N_GAMMA)), None, batch=32, all_momenta=True, verify=False)
    torch.cuda.synchronize()
    print(json.dumps({"fft_only": {"lattice": list(DIMS), "lp_sources": 64, "ms": (time.perf_counter() - t0) * 1e3}}),
          flush=True)
    ctx.close()


def run_dslash_only(tiers):
    import torch
    from paper_1211_0126_gb300 import build, tsm
    from paper_1211_0126_gb300 import synthetic as S
    if not os.path.exists(tsm.LIB_PATH):
        build.build()
    stream = torch.cuda.current_stream()
    ctx = tsm.Context(0, stream.cuda_stream)
    ctx.load_gauge(S.gauge_field(DIMS, EPS, GAUGE_SEED), DIMS, KAPPA, MU)
    psi = S.random_spinor(DIMS, 99)
    out = np.zeros_like(psi)
    names = {"f64": tsm.TSM_F64, "f32": tsm.TSM_F32, "f16": tsm.TSM_F16, "bf16": tsm.TSM_BF16}
    res = {}
    for name in tiers.split(","):
        tsm.tsm_profile(ctx.h, True)
        for _ in range(3):
            tsm.tm_dslash(ctx.h, names[name], tsm.TM_OP_HOP_EO, 0, psi, out)
        ms, cnt, by = ctx.profile_read()
        tsm.tsm_profile(ctx.h, False)
        res[name] = {"us_per_launch": 1e3 * ms.sum() / cnt.sum(), "gbs": by.sum() / (ms.sum() * 1e-3) / 1e9}
    print(json.dumps({"dslash_only": res}), flush=True)
    ctx.close()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle sample
def oracle_sample(U, t_src_too=True):
    """Time the CPU oracle on a bounded sample of the workload: one CG iteration
    (Dhat then Dhat^dag plus the vector updates) at 24^3 x 48 and, optionally,
    the per-source work outside the iterations (Schur source, odd-site
    reconstruction, contraction)."""
    from oracle import dirac, loops, philox
    eta = philox.noise(1000, 0, DIMS, 4)
    e = dirac.even_mask(DIMS)
    p = e * eta
    t0 = time.perf_counter()
    q = dirac.schur(U, p, DIMS, KAPPA, MU)
    alpha = np.vdot(p, p).real / np.vdot(q, q).real
    x = alpha * p
    r = p - alpha * dirac.schur_dag(U, q, DIMS, KAPPA, MU)
    beta = np.vdot(r, r).real / np.vdot(p, p).real
    p = r + beta * p
    t_it = time.perf_counter() - t0
    t_src = None
    if t_src_too:
        t0 = time.perf_counter()
        bh = dirac.schur_source(U, eta, DIMS, KAPPA, MU)
        s = dirac.schur_reconstruct(U, x, eta, DIMS, KAPPA, MU)
        loops.local_loops(eta, s, DIMS, list(range(N_GAMMA)), default_moms())
        # Dhat^dag bhat that starts every solve
        dirac.schur_dag(U, bh, DIMS, KAPPA, MU)
        t_src = time.perf_counter() - t0
    return t_it, t_src


# ------------------------------------------------------------------ the oracle on every host core
_WORKER_U = None


def _oracle_worker_init():
    """Spawned worker: its own copy of the workload's links (same seed)."""
    global _WORKER_U
    from paper_1211_0126_gb300 import synthetic as S
    _WORKER_U = S.gauge_field(DIMS, EPS, GAUGE_SEED)


def _oracle_worker(t_src_too):
    return oracle_sample(_WORKER_U, t_src_too)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The oracle's bounded sample run on every host core at once: one spawned
    worker process per core (spawn, so that no CUDA state is inherited), each
    timing its own sample; the host's throughput is the sum of the workers'
    rates, measured while all of them run.  A worker that dies or a sample
    that overruns `timeout` seconds raises instead of hanging."""

    def __init__(self, cores=None, timeout=300.0):
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        self.cores = cores or host_cores()
        self.timeout = timeout
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"   # one thread per worker: the workers are the parallelism
        self.ex = ProcessPoolExecutor(max_workers=self.cores, mp_context=mp.get_context("spawn"),
                                      initializer=_oracle_worker_init)

    def sample(self, t_src_too=True):
        futs = [self.ex.submit(_oracle_worker, t_src_too) for _ in range(self.cores)]
        return [f.result(timeout=self.timeout) for f in futs]

    def close(self):
        self.ex.shutdown(wait=False, cancel_futures=True)


def oracle_on_host(U, t_src_too=True):
    """(per-worker samples, cores): every host core if the worker pool runs,
    else one sample in this process."""
    pool = None
    try:
        pool = OraclePool()
        res = pool.sample(t_src_too)
        return res, pool
    except Exception as e:   # a broken or overrunning pool: fall back to one core
        print("oracle worker pool unavailable (%s); timing one core" % type(e).__name__, file=sys.stderr)
        if pool is not None:
            pool.close()
        return [oracle_sample(U, t_src_too)], None


def default_moms():
    from paper_1211_0126_gb300 import synthetic as S
    return S.default_momenta(N_Q)


def oracle_rate(t_it, t_src, lp_iters_per_src, hp_iters_per_src):
    """sources/s of the oracle for the workload: every LP solve costs its
    iterations plus the per-source work; every HP-set source adds its HP solve."""
    t_lp = lp_iters_per_src * t_it + t_src
    t_hp = hp_iters_per_src * t_it + t_src
    total = (N_HP + N_LP) * t_lp + N_HP * t_hp
    return (N_HP + N_LP) / total


# HP solves of the oracle: FP64 CG, zero start, the same stopping rule as the
# library's FP64 CG on the same system, hence the same iteration count up to
# rounding.  That count for this workload (24^3 x 48, seed-3 links, Z4 noise,
# 1e-10) is 76, measured by the plain FP64 leg of the GPU arm
# (equal_error.plain_fp64.iters).  A 1e-10 oracle solve at this size (about
# 76 x 14 s on one host core) does not fit a bounded sample; the LP count is
# measured live.
HP_ITERS_FP64_CG = 76


def oracle_lp_source(U, source):
    """One complete LP source of the workload through the oracle's own
    functions: Schur source, CGNR truncated at the LP rule, odd-site
    reconstruction, contraction of 16 Gamma x 7 momenta.  Returns (seconds,
    CG iterations)."""
    from oracle import dirac, loops, philox, solver
    eta = philox.noise(1000, source, DIMS, 4)
    t0 = time.perf_counter()
    bh = dirac.schur_source(U, eta, DIMS, KAPPA, MU)
    xe, iters, _ = solver.cgnr(U, bh, DIMS, KAPPA, MU, LP_TOL, LP_MAXIT)
    s = dirac.schur_reconstruct(U, xe, eta, DIMS, KAPPA, MU)
    loops.local_loops(eta, s, DIMS, list(range(N_GAMMA)), default_moms())
    return time.perf_counter() - t0, int(iters)


def _oracle_lp_worker(source):
    return oracle_lp_source(_WORKER_U, source)


def oracle_schur_apply(U):
    """One application of the oracle's Schur operator Dhat at 24^3 x 48 (half
    of a CG iteration, which applies Dhat and Dhat^dag); seconds."""
    from oracle import dirac, philox
    p = dirac.even_mask(DIMS) * philox.noise(1000, 0, DIMS, 4)
    t0 = time.perf_counter()
    dirac.schur(U, p, DIMS, KAPPA, MU)
    return time.perf_counter() - t0


def _oracle_schur_worker(_):
    return oracle_schur_apply(_WORKER_U)


def base_config():
    """The workload both arms run (the reference arm's line carries the same dict)."""
    return {"workload": WORKLOAD, "lattice": list(DIMS), "n_hp_per_gpu": N_HP, "n_lp_per_gpu": N_LP,
            "noise": "Z4", "hp_stop": [HP_TOL, HP_MAXIT], "lp_stop": [LP_TOL, LP_MAXIT],
            "n_gamma": N_GAMMA, "n_q": N_Q, "l2": "flushed between steps (256 MB write)"}


def run_reference(args):
    """The CPU oracle on the workload, on every host core at once.  Warm-up
    step 0: every worker runs one complete LP source (a different noise
    source each), which measures the LP iteration count and the time of one
    LP source.  Every other step: every worker times one application of the
    Schur operator of the workload; one CG iteration = two of them (Dhat,
    Dhat^dag; the vector updates are a small fraction).  sources/s = 264
    sources / (264 LP sources + 8 HP solves, an HP solve being an LP source
    plus HP_ITERS_FP64_CG - LP iterations more), summed over the workers;
    ms_per_step is the wall time of one timed step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1211_0126_gb300 import synthetic as S
    U, pool = None, None
    try:
        pool = OraclePool()
        ncores = pool.cores
        futs = [pool.ex.submit(_oracle_lp_worker, w) for w in range(ncores)]
        lp = [f.result(timeout=1800.0) for f in futs]
    except Exception as e:   # no worker pool: this process, one core
        print("oracle worker pool unavailable (%s); timing one core" % type(e).__name__, file=sys.stderr)
        if pool is not None:
            pool.close()
        pool = None
        U = S.gauge_field(DIMS, EPS, GAUGE_SEED)
        lp = [oracle_lp_source(U, 0)]
    ncores = len(lp)
    t_lp = np.array([t for t, _ in lp])
    lp_iters = float(np.mean([it for _, it in lp]))
    def one_step():
        if pool is None:
            return [oracle_schur_apply(U)]
        futs = [pool.ex.submit(_oracle_schur_worker, w) for w in range(ncores)]
        return [f.result(timeout=pool.timeout) for f in futs]

    times, walls = [], []   # per timed step: every worker's Schur time, and the step's wall time
    try:
        for k in range(1, args.warmup + args.steps):
            t0 = time.perf_counter()
            res = one_step()
            if k >= args.warmup:
                times.append(res)
                walls.append(time.perf_counter() - t0)
    except Exception as e:   # a worker lost mid-run: report the steps that completed
        print("oracle step failed (%s)" % type(e).__name__, file=sys.stderr)
    if not times:
        times.append(one_step())
    if pool is not None:
        pool.close()
    t_it = 2.0 * np.mean(np.asarray(times), axis=0)   # per worker: Dhat + Dhat^dag
    rate = []
    for w in range(ncores):
        t_hp = t_lp[w] + max(HP_ITERS_FP64_CG - lp_iters, 0.0) * t_it[w]
        rate.append((N_HP + N_LP) / ((N_HP + N_LP) * t_lp[w] + N_HP * t_hp))
    value = float(sum(rate))
    ms_step = 1e3 * float(np.mean(walls)) if walls else None
    sample = ("warm-up: one complete oracle LP source (Schur source, CGNR to %g, reconstruction, 16x7 "
              "contraction) on each of %d worker processes at once: %.1f s, %.2f CG iterations (mean); "
              "each step: one oracle Schur application at 24^3x48 on every worker, a CG iteration being two "
              "(mean iteration %.2f s); HP solve = LP "
              "source + %d - %.2f more iterations (FP64 CG count of this system); summed over the workers "
              "(extrapolated from the measured per-source and per-iteration times)"
              % (LP_TOL, ncores, float(np.mean(t_lp)), lp_iters, float(np.mean(t_it)), HP_ITERS_FP64_CG,
                 lp_iters))
    line = {"metric": METRIC, "value": value, "unit": "sources/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": base_config(),
            "cpu_baseline": {"value": value, "unit": "sources/s", "cores": ncores, "kind": "oracle",
                             "sample": sample, "lp_iters_per_source": lp_iters,
                             "hp_iters_per_source": HP_ITERS_FP64_CG},
            "e2e": {"value": value, "unit": "sources/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def tune_table(tsm, times):
    """the autotuner's ms per source: width -> block shape (sources x registers) -> ms"""
    return {"w%d" % w: {"t%dr%d" % shape: float(times[i, j]) for j, shape in enumerate(tsm.TILE_SHAPES)}
            for i, w in enumerate((8, 16, 32, 64))}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("dslash.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1211_0126_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per hop launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "hop_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1211_0126_gb300 import build, replicas, tsm
    from paper_1211_0126_gb300 import synthetic as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if not os.path.exists(tsm.LIB_PATH):
        if rank == 0:
            build.build()
        if world > 1:
            dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    U = S.gauge_field(DIMS, EPS, GAUGE_SEED)
    U_pinned = torch.from_numpy(U.view(np.float64).reshape(-1)).pin_memory()
    ctx = tsm.Context(local, stream.cuda_stream)
    ctx.load_gauge(U, DIMS, KAPPA, MU)
    gam, moms = list(range(N_GAMMA)), S.default_momenta(N_Q)
    rdelta = args.reliable_delta if args.reliable_delta else RELIABLE_DELTA
    hp_stop = tsm.stop(HP_TOL, HP_MAXIT, tsm.TSM_F32, reliable=True, reliable_delta=rdelta)
    lp_stop = tsm.stop(LP_TOL, LP_MAXIT, tsm.TSM_F16)
    hp_range, lp_range = replicas.source_ranges(N_HP, N_LP, rank, world)
    # launch shape: autotuned (untimed, before the warm-up) unless a batch width is given
    tune = None
    if args.batch is None:
        best, tile, regs, ttimes = tsm.tsm_tune(ctx.h, lp_stop)
        args.batch = best
        tune = {"batch": best, "tile_sources": tile, "max_regs": regs, "ms_per_source": tune_table(tsm, ttimes)}
    E = N_GAMMA * N_Q * DIMS[3]
    shape = (N_GAMMA, N_Q, DIMS[3])
    d_loops = torch.zeros(shape, dtype=torch.complex128, device=dev)
    d_err = torch.zeros(shape, dtype=torch.float64, device=dev)
    d_pc = torch.zeros((N_HP,) + shape, dtype=torch.complex128, device=dev)
    d_pl = torch.zeros((N_LP,) + shape, dtype=torch.complex128, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2

    def step(seed, verify=False):
        p = tsm.params(seed, 4, hp_range, lp_range, hp_stop, lp_stop, gam, moms, batch=args.batch, verify=verify,
                       hp_warm_start=args.hp_warm_start)
        if args.mode == "graph" and not verify:
            return tsm.tsm_loops_graph([ctx.h], [p], loops=[d_loops], err=[d_err], per_corr=[d_pc],
                                       per_lp=[d_pl])[0]
        return tsm.tsm_loops(ctx.h, p, d_loops, d_err, None, None, d_pc, d_pl)

    warm = None
    for k in range(args.warmup):
        # warm-up steps also recompute every HP solution's true residual in FP64
        warm = step(10_000 + k, verify=True)
    # ---------------- timed region
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    tsm.tsm_profile(ctx.h, True)
    launches0 = ctx.launch_count()
    times, stats = [], []
    pooled = PooledMoments()
    for k in range(args.steps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        stats.append(step(20_000 + k))
        ev1.record(stream)
        barrier()
        times.append(ev0.elapsed_time(ev1))
        pooled.add(d_pc, d_pl)   # after the step's end event: per-source moments of every timed step
    launches = ctx.launch_count() - launches0
    prof_ms, prof_cnt, prof_bytes = ctx.profile_read()
    tsm.tsm_profile(ctx.h, False)
    clk = clocks.stop()
    # ---------------- end of timed region
    step_ms = float(sum(times)) / len(times)
    if world > 1:
        t = torch.tensor([step_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms = float(t.item())
    value = world * (N_HP + N_LP) / (step_ms * 1e-3)

    peak, peak_kind = measured_peaks()
    # dominant kernels: the FP16 hop family K1-K4 of the LP solves (tier 3 buckets)
    dom = slice(12, 16)
    tot_ms, tot_bytes, tot_cnt = float(prof_ms[dom].sum()), float(prof_bytes[dom].sum()), int(prof_cnt[dom].sum())
    achieved = tot_bytes / (tot_ms * 1e-3) / 1e9 if tot_ms > 0 else None
    traffic = ncu_traffic()
    per_kernel = {}
    for b in range(16):
        if prof_cnt[b]:
            per_kernel["%s_%s" % (TIERS[b // 4], KINDS[b % 4])] = {
                "launches_timed": int(prof_cnt[b]), "us_per_launch": 1e3 * prof_ms[b] / prof_cnt[b],
                "algorithmic_gbs": prof_bytes[b] / (prof_ms[b] * 1e-3) / 1e9}
    alg_per_launch = (tot_bytes / tot_cnt) if tot_cnt else None
    # FP32 arithmetic view of the same launches: 1320 flop per source-site of
    # each hop; source-sites recovered from the byte count of each kernel kind
    # (links once per launch + spinor streams per source, as accounted in the library)
    vh = int(np.prod(DIMS)) // 2
    lb, sb = 8 * 12 * 2.0, 24 * 2.0
    streams = {0: 2 * sb, 1: 3 * sb, 2: 2 * sb, 3: 3 * sb + 4 * sb}   # the FP16 tier keeps r and x in FP16
    site_rhs = sum((prof_bytes[12 + k] / vh - prof_cnt[12 + k] * lb) / streams[k] * vh for k in range(4))
    alu_tflops = 1320.0 * site_rhs / (tot_ms * 1e-3) / 1e12 if tot_ms > 0 else None
    # FP32 FMA peak of this GPU, measured now by the library's register-resident FMA loop
    try:
        fp32_peak = tsm.tsm_measure_fma_peak(local, tsm.TSM_F32)
    except tsm.TsmError as e:
        print("FMA peak not measured: %s" % e, file=sys.stderr)
        fp32_peak = None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": (traffic["dram_over_algorithmic"] * alg_per_launch
                            if (traffic and alg_per_launch) else None),
                "traffic_source": ("ncu DRAM/algorithmic ratio of the same kernels at 16^3x32 x 32 sources, "
                                   "scaled to this launch" if traffic else "no capture for this kernel source"),
                "algorithmic_bytes_per_launch": alg_per_launch,
                "alu": {"flop_per_source_site": 1320, "achieved_tflops": alu_tflops, "peak_tflops": fp32_peak,
                        "frac": (alu_tflops / fp32_peak) if (alu_tflops and fp32_peak) else None,
                        "peak_source": "measured in this run: tsm_measure_fma_peak (FP32 FMA loop, 2 flop per "
                                       "FMA; nominal 152 SMs x 128 lanes x 2 x 2.07 GHz = 80.5)"},
                "kernel": "FP16 half-Dslash family K1-K4 of the LP solves (batch %d)" % args.batch,
                "peak_source": ("measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                                else "fallback 6.8 TB/s"),
                "per_kernel": per_kernel}

    st = stats[-1]
    line = {"metric": METRIC, "value": value, "unit": "sources/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": base_config(),
            "run": {"batch": args.batch, "autotuner": tune, "reliable_delta": rdelta,
                    "hp_start": "lp-solution" if args.hp_warm_start else "zero",
                    "mode": args.mode,
                    "lp_iters_per_source": st.lp_iters / float(N_HP + N_LP),
                    "hp_iters_per_source": st.hp_iters / float(N_HP),
                    "hp_max_true_res_warmup": (warm.hp_max_true_res if warm is not None else None)},
            "roofline": roofline, "clocks": clk, "gpu_launches": int(launches)}

    if rank == 0 and not args.no_extras:
        line["dslash"] = dslash_gbs(ctx, S, tsm, flush, peak)
        line["e2e"] = e2e_leg(ctx, tsm, U_pinned, lp_stop, hp_stop, gam, moms, stream, hp_range, lp_range,
                              batch=args.batch, warm=args.hp_warm_start)
        line["precision_vs_fp64"] = precision_leg(ctx, tsm, gam, moms, 20_000 + args.steps - 1, d_loops, d_err,
                                                  hp_range, lp_range, args.batch, stream)
        line["equal_error"] = equal_error(ctx, tsm, gam, moms, pooled, step_ms, stream, args.batch, hp_stop,
                                          lp_stop)
        res, pool = oracle_on_host(U, t_src_too=True)
        if pool is not None:
            pool.close()
        lp_it, hp_it = st.lp_iters / float(N_HP + N_LP), st.hp_iters / float(N_HP)
        cpu_val = sum(oracle_rate(ti, ts, lp_it, hp_it) for ti, ts in res)
        line["cpu_baseline"] = {"value": cpu_val, "unit": "sources/s", "cores": len(res), "kind": "oracle",
                                "sample": "one oracle CG iteration at 24^3x48 (mean %.2f s) + per-source work "
                                          "(mean %.2f s) on each of %d worker processes at once, scaled with this "
                                          "run's LP/HP iteration counts and summed over the workers (extrapolated)"
                                          % (float(np.mean([r[0] for r in res])), float(np.mean([r[1] for r in res])),
                                             len(res))}
    if world > 1:
        # one exchange at the end: per-source loops to every rank, combined in rank order
        g = dist.new_group(backend="gloo")
        pc, pl = replicas.gather_per_source(d_pc.cpu().numpy(), d_pl.cpu().numpy(), g)
        comb = ctx.combine(pc, pl)
        line["combined_sources"] = int(pc.shape[0] + pl.shape[0])
        line["combined_finite"] = bool(np.isfinite(comb["loops"]).all())
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def dslash_gbs(ctx, S, tsm, flush, peak):
    """Standalone H_eo launches per tier at 24^3 x 48, L2 flushed before each
    call; kernel time from CUDA events around the hop launch."""
    psi = S.random_spinor(DIMS, 99)
    out = np.zeros_like(psi)
    res = {}
    for name, prec in (("f64", tsm.TSM_F64), ("f32", tsm.TSM_F32), ("f16", tsm.TSM_F16), ("bf16", tsm.TSM_BF16)):
        for _ in range(2):
            tsm.tm_dslash(ctx.h, prec, tsm.TM_OP_HOP_EO, 0, psi, out)
        tsm.tsm_profile(ctx.h, True)
        for _ in range(10):
            flush.zero_()
            tsm.tm_dslash(ctx.h, prec, tsm.TM_OP_HOP_EO, 0, psi, out)
        ms, cnt, by = ctx.profile_read()
        tsm.tsm_profile(ctx.h, False)
        gbs = by.sum() / (ms.sum() * 1e-3) / 1e9
        t_launch = ms.sum() * 1e-3 / cnt.sum()
        res[name] = {"us_per_launch": 1e6 * t_launch, "algorithmic_gbs": gbs, "frac": gbs / peak,
                     "bytes_per_site": by.sum() / cnt.sum() / (np.prod(DIMS) // 2),
                     # labelled "naive" count (no spinor reuse): 8 links + 8 neighbour spinors + 1
                     # output per site, 312 reals (the FP64 tier stores 18-real links: 360)
                     "naive_gbs": NAIVE_REALS[name] * REAL_BYTES[name] * (np.prod(DIMS) // 2) / t_launch / 1e9}
    # the FP64 stencil is bound by the FP64 pipe on GB300: its arithmetic rate
    # (1320 flop per site) against the FP64 FMA peak measured now
    import torch
    p64 = tsm.tsm_measure_fma_peak(torch.cuda.current_device(), tsm.TSM_F64)
    f64_tflops = 1320.0 * (np.prod(DIMS) // 2) / (res["f64"]["us_per_launch"] * 1e-6) / 1e12
    res["f64"]["alu"] = {"bound": "alu", "achieved_tflops": f64_tflops, "peak_tflops": p64,
                         "frac": f64_tflops / p64, "unit": "TFLOP/s",
                         "peak_source": "measured in this run: tsm_measure_fma_peak (FP64 FMA loop)"}
    return res


def e2e_leg(ctx, tsm, U_pinned, lp_stop, hp_stop, gam, moms, stream, hp_range, lp_range, steps=3, batch=1,
            warm=False, warmup=1):
    """The same TSM step through the public API with host buffers: gauge field
    uploaded from pinned host memory, loops and errors read back to host; host
    wall clock per step, after `warmup` untimed steps of the same kind (the
    first call with host outputs allocates their staging buffers)."""
    import torch
    shape = (N_GAMMA, N_Q, DIMS[3])
    loops = np.zeros(shape, dtype=np.complex128)
    err = np.zeros(shape, dtype=np.float64)
    ms = []
    for k in range(warmup + steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tsm.tsm_load_gauge(ctx.h, ctx.lat, U_pinned)
        p = tsm.params(30_000 + k, 4, hp_range, lp_range, hp_stop, lp_stop, gam, moms, batch=batch,
                       hp_warm_start=warm)
        tsm.tsm_loops(ctx.h, p, loops, err)
        if k >= warmup:
            ms.append((time.perf_counter() - t0) * 1e3)
    t = float(np.mean(ms))
    return {"value": (N_HP + N_LP) / (t * 1e-3), "unit": "sources/s",
            "h2d_bytes_per_step": int(U_pinned.numel() * 8), "d2h_bytes_per_step": int(loops.nbytes + err.nbytes),
            "ms_per_step": t, "steps": steps, "warmup": warmup, "clock": "host wall clock around each step"}


class PooledMoments:
    """Per-entry sums of x and |x|^2 of the per-source loops of every timed
    step (each step draws fresh noise, so the sources of all steps are
    independent samples): HP-set corrections and LP-set loops, per entry and
    summed over t."""

    def __init__(self):
        self.n = [0, 0]
        self.s1 = [None, None]
        self.s2 = [None, None]
        self.t1 = [None, None]
        self.t2 = [None, None]

    def add(self, pc, pl):
        for k, x in enumerate((pc, pl)):
            xt = x.sum(-1)
            parts = (x.sum(0), (x.abs() ** 2).sum(0), xt.sum(0), (xt.abs() ** 2).sum(0))
            if self.s1[k] is None:
                self.s1[k], self.s2[k], self.t1[k], self.t2[k] = parts
            else:
                self.s1[k] += parts[0]
                self.s2[k] += parts[1]
                self.t1[k] += parts[2]
                self.t2[k] += parts[3]
            self.n[k] += x.shape[0]

    def var(self, k, summed_t):
        """unbiased complex sample variance per entry (numpy)"""
        a, b = (self.t1[k], self.t2[k]) if summed_t else (self.s1[k], self.s2[k])
        n = self.n[k]
        return ((b - a.abs() ** 2 / n) / (n - 1)).cpu().numpy()


def precision_leg(ctx, tsm, gam, moms, seed, d_loops, d_err, hp_range, lp_range, batch, stream):
    """Each loop's error against the FP64 path: the last timed step again with
    every solve in FP64 (HP to 1e-10, LP with the same truncation rule), the
    same seed, hence the same noise; |L_mixed - L_FP64| / sigma_FP64 per entry."""
    import torch
    ref_loops, ref_err = torch.zeros_like(d_loops), torch.zeros_like(d_err)
    p = tsm.params(seed, 4, hp_range, lp_range, tsm.stop(HP_TOL, HP_MAXIT, tsm.TSM_F64),
                   tsm.stop(LP_TOL, LP_MAXIT, tsm.TSM_F64), list(gam), moms, batch=batch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tsm.tsm_loops(ctx.h, p, ref_loops, ref_err)
    torch.cuda.synchronize()
    t_fp64 = time.perf_counter() - t0
    dz = ((d_loops - ref_loops).abs() / ref_err).cpu().numpy()
    rel = ((d_loops - ref_loops).abs() / ref_loops.abs().max()).cpu().numpy()
    return {"seed": seed, "reference": "the same TSM step with FP64 HP (1e-10) and FP64 LP (same truncation)",
            "max_abs_diff_over_sigma": float(dz.max()), "median_abs_diff_over_sigma": float(np.median(dz)),
            "max_abs_diff_over_sigma_per_gamma": [float(dz[g].max()) for g in range(dz.shape[0])],
            "max_abs_diff_rel_to_max_loop": float(rel.max()), "bar": 0.1, "fp64_step_s": t_fp64}


def equal_error(ctx, tsm, gam, moms, pooled, step_ms, stream, batch, hp_stop, lp_stop, n_plain=64):
    """TSM against the plain FP64 path at equal loop error (the synthetic
    analogue of the paper's HP/LP tuning, Sec. 2.2 and Fig. 1).

    Plain path: every source solved to 1e-10 in FP64, standard estimator.  Its
    per-source variance sigma_P^2 comes from n_plain plain FP64 solves and its
    per-source cost t_P from single-source solves (tsm_loops with an empty HP
    set, FP64 LP rule 1e-10, batch 1).  TSM: sigma_corr^2 and sigma_LP^2 pooled
    over every timed step; t_LP from an LP-only step (256 sources) and t_HP =
    (step - 264 t_LP) / 8.  With r = N_LP / N_HP = sqrt((sigma_LP^2 / t_LP) /
    (sigma_corr^2 / (t_HP + t_LP))), the cost of error eps is T_TSM = (sigma_corr^2
    + sigma_LP^2 / r) (t_HP + t_LP + r t_LP) / eps^2 against T_P = sigma_P^2 t_P
    / eps^2.  One direct run confirms it: a TSM run sized by r for the plain
    run's error on Gamma = 1, q = 0, sum_t, timed, its wall time scaled to
    exactly that error."""
    import torch
    E = N_GAMMA * N_Q * DIMS[3]
    shape = (N_GAMMA, N_Q, DIMS[3])
    out = {}
    # plain FP64 path: n_plain sources, single-source solves
    plain64 = tsm.stop(HP_TOL, HP_MAXIT, tsm.TSM_F64)
    pl_plain = torch.zeros((n_plain,) + shape, dtype=torch.complex128, device="cuda")
    l_plain, e_plain = torch.zeros(shape, dtype=torch.complex128, device="cuda"), \
        torch.zeros(shape, dtype=torch.float64, device="cuda")
    p = tsm.params(40_000, 4, (0, 0), (0, n_plain), plain64, plain64, list(gam), moms, batch=1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = tsm.tsm_loops(ctx.h, p, l_plain, e_plain, None, None, None, pl_plain)
    e1.record(stream)
    torch.cuda.synchronize()
    T_plain = e0.elapsed_time(e1) * 1e-3
    t_p = T_plain / n_plain
    out["plain_fp64"] = {"sources": n_plain, "s_per_source": t_p, "iters": st.lp_iters / float(n_plain)}
    # LP-only step for t_LP
    lp_only = tsm.params(40_100, 4, (0, 0), (0, N_LP), hp_stop, lp_stop, list(gam), moms, batch=batch)
    tsm.tsm_loops(ctx.h, lp_only, l_plain, e_plain)   # warm
    torch.cuda.synchronize()
    e0.record(stream)
    tsm.tsm_loops(ctx.h, lp_only, l_plain, e_plain)
    e1.record(stream)
    torch.cuda.synchronize()
    t_lp = e0.elapsed_time(e1) * 1e-3 / N_LP
    t_hp = max((step_ms * 1e-3 - (N_HP + N_LP) * t_lp) / N_HP, 1e-9)
    out["tsm_costs"] = {"t_lp_s": t_lp, "t_hp_s": t_hp, "pooled_hp_sources": pooled.n[0],
                        "pooled_lp_sources": pooled.n[1]}
    xp = pl_plain.cpu().numpy()

    def var_np(x):
        return np.var(x.real, axis=0, ddof=1) + np.var(x.imag, axis=0, ddof=1)

    vp_all, vp_t = var_np(xp), var_np(xp.sum(-1))
    vc_all, vc_t = pooled.var(0, False), pooled.var(0, True)
    vl_all, vl_t = pooled.var(1, False), pooled.var(1, True)

    def ratio(vp, vc, vl):
        r = np.sqrt((vl / t_lp) / (vc / (t_hp + t_lp)))
        t_tsm = (vc + vl / r) * (t_hp + t_lp + r * t_lp)   # x eps^2
        fixed = (vc / N_HP + vl / N_LP) * (step_ms * 1e-3)   # x eps^2 with this run's allocation
        return r, vp * t_p / t_tsm, vp * t_p / fixed, vp / t_tsm

    sel = {"Gamma=1,q=0,sum_t": 0, "Gamma=gamma3gamma5,q=0,sum_t": 8}
    for name, g in sel.items():
        r, rat, rat_fixed, eff = ratio(vp_t[g, 0], vc_t[g, 0], vl_t[g, 0])
        out[name] = {"sigma2_plain": float(vp_t[g, 0]), "sigma2_corr": float(vc_t[g, 0]),
                     "sigma2_lp": float(vl_t[g, 0]), "optimal_n_lp_over_n_hp": float(r),
                     "ratio_vs_plain_fp64": float(rat), "ratio_at_this_runs_allocation": float(rat_fixed),
                     "tsm_effective_sources_per_s": float(eff), "plain_sources_per_s": 1.0 / t_p}
    ok = (vl_all > 0) & (vc_all > 0) & (vp_all > 0)
    r_all = np.sqrt((vl_all[ok] / t_lp) / (vc_all[ok] / (t_hp + t_lp)))
    rat_all = vp_all[ok] * t_p / ((vc_all[ok] + vl_all[ok] / r_all) * (t_hp + t_lp + r_all * t_lp))
    out["median_all_entries_ratio_vs_plain_fp64"] = float(np.median(rat_all))
    # direct confirmation on Gamma = 1, q = 0, sum_t at the plain run's error
    g = 0
    eps_p = float(np.sqrt(vp_t[g, 0] / n_plain))
    r = out["Gamma=1,q=0,sum_t"]["optimal_n_lp_over_n_hp"]
    n_hp = max(2, int(np.ceil((vc_t[g, 0] + vl_t[g, 0] / r) / eps_p ** 2)))
    n_lp = max(2, int(round(r * n_hp)))
    d_l = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    d_c = torch.zeros((n_hp,) + shape, dtype=torch.complex128, device="cuda")
    d_p = torch.zeros((n_lp,) + shape, dtype=torch.complex128, device="cuda")
    pd = tsm.params(50_000, 4, (0, n_hp), (n_hp, n_hp + n_lp), hp_stop, lp_stop, list(gam), moms, batch=batch)
    torch.cuda.synchronize()
    e0.record(stream)
    tsm.tsm_loops(ctx.h, pd, d_l, None, None, None, d_c, d_p)
    e1.record(stream)
    torch.cuda.synchronize()
    T_tsm = e0.elapsed_time(e1) * 1e-3
    c = d_c.cpu().numpy().sum(-1)[:, g, 0]
    lv = d_p.cpu().numpy().sum(-1)[:, g, 0]
    eps_tsm = float(np.sqrt((np.var(c.real, ddof=1) + np.var(c.imag, ddof=1)) / n_hp +
                            (np.var(lv.real, ddof=1) + np.var(lv.imag, ddof=1)) / n_lp))
    T_tsm_eq = T_tsm * (eps_tsm / eps_p) ** 2
    out["direct_confirmation"] = {"loop": "Gamma=1,q=0,sum_t", "plain_sources": n_plain, "plain_s": T_plain,
                                  "plain_error": eps_p, "tsm_n_hp": n_hp, "tsm_n_lp": n_lp, "tsm_s": T_tsm,
                                  "tsm_error": eps_tsm, "tsm_s_at_plain_error": T_tsm_eq,
                                  "ratio_vs_plain_fp64": T_plain / T_tsm_eq}
    return out


def run_three_lattice(args):
    """Batching workload: three lattices (8^3x16, 12^3x24, 16^3x32; links
    eps = 0.25, kappa = 0.1245, mu = 0.005), per lattice N_LP = 512 BF16 LP
    solves at 1e-2 and N_HP = 16 FP32+FP64 HP solves at 1e-10, batch widths
    from the autotuner, all three TSM estimates in one captured CUDA graph.
    Reports sources/s of the graph and of the same work run eagerly."""
    import torch
    from paper_1211_0126_gb300 import build, tsm
    from paper_1211_0126_gb300 import synthetic as S
    if not os.path.exists(tsm.LIB_PATH):
        build.build()
    lattices = [(8, 8, 8, 16), (12, 12, 12, 24), (16, 16, 16, 32)]
    n_hp, n_lp = 16, 512
    hp = tsm.stop(1e-10, HP_MAXIT, tsm.TSM_F32, reliable=True, reliable_delta=RELIABLE_DELTA)
    lp = tsm.stop(1e-2, 500, tsm.TSM_BF16)
    gam, moms = list(range(N_GAMMA)), S.default_momenta(N_Q)
    ctxs, widths, tune = [], [], {}
    for k, dims in enumerate(lattices):
        ctx = tsm.Context(0)
        ctx.load_gauge(S.gauge_field(dims, EPS, 100 + k), dims, KAPPA, MU)
        best, tile, regs, times = tsm.tsm_tune(ctx.h, lp)
        ctxs.append(ctx)
        widths.append(best)
        tune["x".join(map(str, dims))] = {"batch": best, "tile_sources": tile, "max_regs": regs,
                                          "ms_per_source": tune_table(tsm, times)}
    outs = [torch.zeros((len(gam), len(moms), d[3]), dtype=torch.complex128, device="cuda") for d in lattices]

    def plist(seed):
        return [tsm.params(seed + k, 4, (0, n_hp), (n_hp, n_hp + n_lp), hp, lp, gam, moms, batch=widths[k])
                for k in range(len(lattices))]

    def graph_step(seed):
        return tsm.tsm_loops_graph([c.h for c in ctxs], plist(seed), loops=outs)

    def eager_step(seed):
        for k, c in enumerate(ctxs):
            tsm.tsm_loops(c.h, plist(seed)[k], outs[k])

    res = {}
    for name, fn in (("graph", graph_step), ("eager", eager_step)):
        for w in range(args.warmup):
            fn(1000 + w)
        torch.cuda.synchronize()
        ms = []
        for k in range(args.steps):
            t0 = time.perf_counter()
            fn(2000 + k)
            torch.cuda.synchronize()
            ms.append((time.perf_counter() - t0) * 1e3)
        res[name] = {"ms_per_step": float(np.mean(ms)),
                     "sources_per_s": 3 * (n_hp + n_lp) / (float(np.mean(ms)) * 1e-3)}
    st = graph_step(3000)
    line = {"metric": "TSM sources/sec, three lattices in one captured graph", "value": res["graph"]["sources_per_s"],
            "unit": "sources/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["graph"]["ms_per_step"], "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "three-lattice 8^3x16+12^3x24+16^3x32, per lattice hp16(f32+f64rel,1e-10) "
                                   "lp512(bf16,1e-2)", "autotune": tune,
                       "lp_iters_per_source": [s.lp_iters / float(n_hp + n_lp) for s in st],
                       "hp_iters_per_source": [s.hp_iters / float(n_hp) for s in st]},
            "eager": res["eager"], "graph_speedup": res["eager"]["ms_per_step"] / res["graph"]["ms_per_step"]}
    print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()


def run_learned(args):
    """Learned-preconditioner workload: 16^3x32, links eps = 0.25 (seeds 201-204
    train, 205-206 held out), kappa = 0.1245, mu = 0.005.  A 4-layer
    parallel-transport network (channels 1-12-12-12-1, BF16 channel mixing on
    the tensor cores) is trained with Adam on 4 x pairs-per-field (r, Dhat^-1 r)
    pairs, once on white Z4 noise with FP32 CG targets (1e-6) and once on the
    Krylov residuals of the training fields' own FP32 CGNR solves (iterations
    0, 1, 2, 4, 8, targets x* - x_k), and evaluated on the held-out fields:
    relative loss; flexible GMRES with the trained and with the untrained
    (near-identity) network against CG at the LP tolerance 1e-2; and the TSM
    estimate with N_HP = 16, N_LP = 1024 using learned LP solves (the network
    whose flexible GMRES is cheaper) against plain BF16 CG LP solves, compared
    at equal loop error (time x variance)."""
    import torch
    from paper_1211_0126_gb300 import build, tsm
    from paper_1211_0126_gb300 import synthetic as S
    if not os.path.exists(tsm.LIB_PATH):
        build.build()
    dims = (16, 16, 16, 32)
    channels = [1, 12, 12, 12, 1]
    gam, moms = list(range(N_GAMMA)), S.default_momenta(N_Q)
    pair_stop = tsm.stop(1e-6, 4000, tsm.TSM_F32)
    lp_cg = tsm.stop(1e-2, 500, tsm.TSM_BF16)
    lp_fg = tsm.stop(1e-2, 500, tsm.TSM_BF16, precond=True, restart=16)
    hp = tsm.stop(1e-10, HP_MAXIT, tsm.TSM_F32, reliable=True, reliable_delta=RELIABLE_DELTA)
    ctxs = []
    for seed in range(201, 207):
        c = tsm.Context(0)
        c.load_gauge(S.gauge_field(dims, EPS, seed), dims, KAPPA, MU)
        ctxs.append(c)
    train, held = ctxs[:4], ctxs[4:]
    untrained = tsm.Network(channels, seed=7, init_scale=0.1)
    its = [0, 1, 2, 4, 8]

    def trained_net(kind):
        """a network trained on one kind of pairs, its held-out losses and timings"""
        model = tsm.Network(channels, seed=7, init_scale=0.1)
        t0 = time.perf_counter()
        if kind == "solves":
            g_tr = [model.add_solve_pairs(c, max(1, args.pairs_per_field // len(its)), 300 + k, its, pair_stop)
                    for k, c in enumerate(train)]
            g_he = [model.add_solve_pairs(c, 8, 400 + k, its, pair_stop) for k, c in enumerate(held)]
        else:
            g_tr = [model.add_pairs(c, args.pairs_per_field, 300 + k, pair_stop) for k, c in enumerate(train)]
            g_he = [model.add_pairs(c, 32, 400 + k, pair_stop) for k, c in enumerate(held)]
        torch.cuda.synchronize()
        t_pairs = time.perf_counter() - t0
        loss0 = [model.loss(g) for g in g_he]
        t0 = time.perf_counter()
        hist = model.train(g_tr, args.train_steps, 4, 2e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        loss1 = [model.loss(g) for g in g_he]
        info = {"pairs": ("Krylov residuals of the fields' own FP32 CGNR solves at iterations %s (targets "
                          "x* - x_k; k = 0: the source)" % its) if kind == "solves"
                else "white Z4 noise on even sites, FP32 CG targets",
                "pairs_s": t_pairs, "train_s": t_train,
                "train_ms_per_step": t_train * 1e3 / max(args.train_steps, 1),
                "train_loss_first_last": [float(np.mean(hist[:10])), float(np.mean(hist[-10:]))],
                "heldout_loss_before_after": [float(np.mean(loss0)), float(np.mean(loss1))]}
        print("learned (%s pairs): pairs %.1f s, training %.1f s, held-out loss %.4f -> %.4f"
              % (kind, t_pairs, t_train, float(np.mean(loss0)), float(np.mean(loss1))), file=sys.stderr, flush=True)
        return model, info

    def solve_stats(c, stp, model, n=16):
        c.set_precond(model)
        b = np.stack([c.noise(900, j) for j in range(n)])
        c.solve(b[:2], stp)
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, it, tr, _ = c.solve(b, stp)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t) * 1e3 / n
        c.set_precond(None)
        return {"iters": float(np.mean(it)), "true_res": float(np.mean(tr)), "ms_per_solve": ms}

    nets, infos = {}, {}
    for kind in ("noise", "solves"):
        nets[kind], infos[kind] = trained_net(kind)
    solves = {"cg_bf16": [solve_stats(c, lp_cg, None) for c in held],
              "fgmres_untrained": [solve_stats(c, lp_fg, untrained) for c in held]}
    for kind in ("noise", "solves"):
        solves["fgmres_trained_" + kind] = [solve_stats(c, lp_fg, nets[kind]) for c in held]
    print("learned: solves at 1e-2 %s" % json.dumps(solves), file=sys.stderr, flush=True)
    # the TSM comparison uses the network whose flexible GMRES is cheaper per solve
    best_kind = min(("noise", "solves"),
                    key=lambda k: np.mean([s["ms_per_solve"] for s in solves["fgmres_trained_" + k]]))
    net = nets[best_kind]
    tsm_cmp = []
    for k, c in enumerate(held):
        row = {}
        for name, lp, model in (("plain_cg", lp_cg, None), ("learned", lp_fg, net)):
            c.set_precond(model)
            c.loops(50 + k, 4, 2, 8, hp, lp, gam, moms, batch=32)     # warm-up
            torch.cuda.synchronize()
            t = time.perf_counter()
            out = c.loops(60 + k, 4, 16, 1024, hp, lp, gam, moms, batch=32)
            torch.cuda.synchronize()
            row[name] = {"s": time.perf_counter() - t, "err2": out["err"] ** 2,
                         "lp_iters_per_source": out["stats"]["lp_iters"] / 1040.0}
            print("learned: TSM field %d %s %.1f s" % (k, name, row[name]["s"]), file=sys.stderr, flush=True)
            c.set_precond(None)
        ok = row["plain_cg"]["err2"] > 0
        var = row["learned"]["err2"][ok] / row["plain_cg"]["err2"][ok]
        ratio = var * row["learned"]["s"] / row["plain_cg"]["s"]
        tsm_cmp.append({"plain_cg_s": row["plain_cg"]["s"], "learned_s": row["learned"]["s"],
                        "plain_lp_iters": row["plain_cg"]["lp_iters_per_source"],
                        "learned_lp_iters": row["learned"]["lp_iters_per_source"],
                        "median_var_ratio": float(np.median(var)),
                        "median_cost_at_equal_error_ratio": float(np.median(ratio))})
    gain = float(np.mean([r["median_cost_at_equal_error_ratio"] for r in tsm_cmp]))
    line = {"metric": "learned LP preconditioner: TSM cost at equal loop error, learned / plain CG",
            "value": gain, "unit": "ratio (<1: learned cheaper)", "n_gpus": 1, "higher_is_better": False,
            "data": "synthetic",
            "config": {"workload": "learned-16^3x32-eps0.25-k0.1245-mu0.005 net1-12-12-12-1 "
                                   "train 4 fields x %d pairs, held-out 2 fields; TSM hp16 lp1024 at 1e-2"
                                   % args.pairs_per_field,
                       "train_steps": args.train_steps, "batch": 4, "lr": 2e-3},
            "training": infos, "tsm_network": best_kind,
            "solves_at_1e-2": solves, "tsm_equal_error": tsm_cmp}
    print(json.dumps(line), flush=True)
    for m in nets.values():
        m.close()
    untrained.close()
    for c in ctxs:
        c.close()


def run_scale(args):
    """TSM at scale: 32^3x64, links eps = 0.2 after 2 APE steps (alpha = 0.5,
    seed 301), kappa = 0.1248, mu = 0.003; N_HP = 32 FP32 + FP64-reliable solves
    at 1e-10, N_LP = 2048 BF16 solves at 1e-2, blocks of 16 sources; 16 local
    insertions plus the one-derivative insertions along all four directions at
    13 momenta.  One timed step after a smaller warm-up (oracle spot checks of
    sources at this size are GPU tests, not part of the bench)."""
    import torch
    from paper_1211_0126_gb300 import build, tsm
    from paper_1211_0126_gb300 import synthetic as S
    if not os.path.exists(tsm.LIB_PATH):
        build.build()
    dims = (32, 32, 32, 64)
    kappa, mu = 0.1248, 0.003
    n_hp, n_lp = 32, 2048
    gam, moms = list(range(16)), S.default_momenta(13)
    U = S.gauge_field(dims, 0.2, 301, ape_steps=2, ape_alpha=0.5)
    stream = torch.cuda.current_stream()
    ctx = tsm.Context(0, stream.cuda_stream)
    ctx.load_gauge(U, dims, kappa, mu)
    hp = tsm.stop(1e-10, HP_MAXIT, tsm.TSM_F32, reliable=True, reliable_delta=RELIABLE_DELTA)
    lp = tsm.stop(1e-2, 500, tsm.TSM_BF16)
    ctx.loops(5, 4, 2, 16, hp, lp, gam, moms, batch=16, deriv_mask=0b1111)     # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0.record(stream)
    out = ctx.loops(6, 4, n_hp, n_lp, hp, lp, gam, moms, batch=16, deriv_mask=0b1111)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    st = out["stats"]
    line = {"metric": "TSM sources/s at 32^3x64 with local and one-derivative insertions",
            "value": (n_hp + n_lp) / (ms * 1e-3), "unit": "sources/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": ms, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "scale-32^3x64-eps0.2-ape2-k0.1248-mu0.003 hp32(f32+f64rel,1e-10) "
                                   "lp2048(bf16,1e-2) batch16 16G+4 derivative directions x 13q",
                       "lp_iters_per_source": st["lp_iters"] / float(n_hp + n_lp),
                       "hp_iters_per_source": st["hp_iters"] / float(n_hp),
                       "hp_not_converged": st["hp_not_converged"], "hp_max_true_res": st["hp_max_true_res"],
                       "verify": "every HP solution's true residual recomputed in FP64"},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_estimators(args):
    """Every estimator of the path on the 24^3x48 workload (the same 8 HP + 256
    LP solves, 16 Gamma x 7 momenta): the standard one, the one-end trick
    (Eq. 2.5), the generalised one-end trick (Eq. 2.6, one Wilson application
    per solution), the one-derivative insertions along all four directions,
    and all spatial momenta through the library's 3-D FFT.  Per estimator: the
    step time (CUDA events, L2 flushed between steps) and, from one
    instrumented step, the estimator's own kernels (contraction passes,
    derivative passes, FFT projection, Wilson application) with their
    algorithmic bytes against the measured HBM peak."""
    import torch
    from paper_1211_0126_gb300 import build, tsm
    from paper_1211_0126_gb300 import synthetic as S
    if not os.path.exists(tsm.LIB_PATH):
        build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = measured_peaks()
    U = S.gauge_field(DIMS, EPS, GAUGE_SEED)
    ctx = tsm.Context(0, stream.cuda_stream)
    ctx.load_gauge(U, DIMS, KAPPA, MU)
    gam, moms = list(range(N_GAMMA)), S.default_momenta(N_Q)
    hp_stop = tsm.stop(HP_TOL, HP_MAXIT, tsm.TSM_F32, reliable=True, reliable_delta=RELIABLE_DELTA)
    lp_stop = tsm.stop(LP_TOL, LP_MAXIT, tsm.TSM_F16)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2
    variants = [("standard", {}), ("one_end", {"estimator": 1}), ("gen_one_end", {"estimator": 2}),
                ("derivative_4_directions", {"deriv_mask": 0b1111}), ("all_momenta_fft", {"all_momenta": True})]
    buckets = {tsm.PB_CONTRACT: "contraction", tsm.PB_DERIV: "derivative_contraction", tsm.PB_FFT: "fft_projection",
               tsm.PB_WILSON: "wilson_application"}
    clocks = ClockSampler(0)
    clocks.start()
    results = {}
    for name, kw in variants:
        if kw.get("all_momenta"):
            shape, mom = (N_GAMMA, DIMS[3], DIMS[2], DIMS[1], DIMS[0]), [(0, 0, 0)]
            pc = pl = None
        else:
            nblk = 1 + bin(kw.get("deriv_mask", 0)).count("1")
            shape, mom = ((nblk,) if nblk > 1 else ()) + (N_GAMMA, N_Q, DIMS[3]), moms
            pc = torch.zeros((N_HP,) + shape, dtype=torch.complex128, device=dev)
            pl = torch.zeros((N_LP,) + shape, dtype=torch.complex128, device=dev)
        d_loops = torch.zeros(shape, dtype=torch.complex128, device=dev)
        d_err = torch.zeros(shape, dtype=torch.float64, device=dev)

        def step(seed):
            p = tsm.params(seed, 4, (0, N_HP), (N_HP, N_HP + N_LP), hp_stop, lp_stop, gam, mom, batch=args.batch or 32,
                           **kw)
            return tsm.tsm_loops(ctx.h, p, d_loops, d_err, None, None, pc, pl)

        for k in range(args.warmup):
            step(100 + k)
        times = []
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(200 + k)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        tsm.tsm_profile(ctx.h, True)
        step(300)
        bms, bcnt, bby = ctx.profile_read_ex()
        tsm.tsm_profile(ctx.h, False)
        kern = {}
        for b, label in buckets.items():
            if bcnt[b] > 0 and bms[b] > 0:
                gbs = bby[b] / (bms[b] * 1e-3) / 1e9
                kern[label] = {"calls": int(bcnt[b]), "us_per_call": 1e3 * bms[b] / bcnt[b],
                               "algorithmic_bytes_per_call": bby[b] / bcnt[b], "algorithmic_gbs": gbs,
                               "frac": gbs / peak}
        ms = float(np.mean(times))
        results[name] = {"ms_per_step": ms, "sources_per_s": (N_HP + N_LP) / (ms * 1e-3),
                         "output_entries": int(np.prod(shape)), "kernels": kern}
    clk = clocks.stop()
    line = {"metric": "TSM sources/s per estimator at 24^3x48 (the same solves; estimator-specific contraction)",
            "value": results["standard"]["sources_per_s"], "unit": "sources/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"workload": WORKLOAD + " x {standard, one-end, generalised one-end, 4 derivative "
                                              "directions, all momenta by FFT}",
                       "l2": "flushed between steps (256 MB write)",
                       "peak": {"hbm_gbs": peak, "source": peak_kind}},
            "estimators": results, "clocks": clk}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.net_only:
        run_net_only()
    elif args.lp_only:
        run_lp_only()
    elif args.fft_only:
        run_fft_only()
    elif args.contract_only:
        run_contract_only()
    elif args.dslash_only:
        run_dslash_only(args.dslash_only)
    elif args.workload == "three-lattice":
        run_three_lattice(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "scale":
        run_scale(args)
    elif args.workload == "estimators":
        run_estimators(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
