"""Benchmark: SA spin-flip attempts/s and SPVAR TTS99 of Multi-start SPVAR
(Alg. 2), batched against plain form, on one GB300.

The headline workload is a Chimera C8 +-J problem (N = 512, 1472 couplers,
h = 0): 10 starts x (1000 fixing + 1000 solving) samples, 1000 sweeps,
geometric beta 0.1 -> 3.0, elite 10 %, fixing threshold 1.  One step = one
full Multi-start SPVAR run (every start: sample, elite, persistence,
fold/compact, solving sample) through the C-ABI library.  ``value`` is
attempts/s of the batched form (persistent sweep + CUDA graph) with the
problem resident on the device; ``plain`` is the one-launch-per-start form;
``e2e`` goes through spvar_problem_create + spvar_solve with host buffers.

Every sweep kernel's roofline divides its algorithmic integer operations per
second by the measured issue ceiling of this GPU (spvar_measure_issue_rate:
lop3 and mad.lo chains on both integer pipes), and the wide-multiply ceiling
(mul.wide chains) bounds the Philox part.  TTS99 (Sec. III.A R99 in wall time)
is measured on a 3D +-J L = 12 problem at 1000 sweeps, where the per-start
success rate lies strictly between 0 and 1, against a best-known energy from
independent long runs (PTICM at 10^4 sweeps and SA at 2 x 10^4 sweeps), for
SA alone, SPVAR batched, SPVAR plain and the oracle solving on the host cores.
``--impl reference`` times the oracle on the host cores instead.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SA spin-flip attempts/s (SPVAR TTS99 beside it), batched vs plain form"
UNIT = "spin-flip attempts/s"
WORKLOAD = dict(workload="Chimera C8 +-J N=512 h=0 (seed 1200): 10 starts x (1000+1000) samples, 1000 sweeps, "
                         "beta 0.1->3, elite 0.1")
INSTANCE_SEED = 1200
RUN_SEED0 = 42
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
PHILOX_OPS_PER_ATTEMPT = 15  # 10 rounds x (2 wide multiplies + 2 three-input xors + 2 key adds) / 4 replicas
ACCEPT_OPS_PER_ATTEMPT = 3   # dE, dE <= 0 test, threshold compare
WIDE_PER_ATTEMPT = 15 / 4    # wide multiplies per attempt left after the kernels hoist the item-constant ones
# TTS99 workload: 3D +-J L = 12 (one of the uneven batch's sizes), Table II's sample split
TTS_L, TTS_SEED, TTS_T, TTS_STARTS, TTS_S, TTS_ELITE = 12, 1612, 1000, 200, 250, 0.2
TTS_RUN_SEED = 1700


def r4(x):
    """Four significant digits (keeps the line short enough for the driver's tail)."""
    if isinstance(x, float):
        return float("%.4g" % x) if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: r4(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [r4(v) for v in x]
    return x


def _instance():
    from paper_1706_07826_gb300 import instances as I
    return I.chimera(8, INSTANCE_SEED)


def _params(form, rank=0):
    from paper_1706_07826_gb300 import spvar
    # rank r runs global starts 10r .. 10r+9 (weak scaling, no data-path collective)
    return spvar.make_params(num_starts=10, fixing_sample_size=1000, solving_sample_size=1000, num_sweeps=1000,
                             beta0=0.1, beta1=3.0, elite_threshold=0.1, fix_num=1, fix_den=1, iterate=False,
                             max_fix_phases=1, canon=-1, form=form, start_offset=10 * rank)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        load = [x for x in sm if x > 0.5 * mx] if mx else sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------- CPU baseline
def _oracle_worker(args):
    r0, R = args
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    inst = _instance()
    p = O.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J, inst.h)
    thr = O.thresholds(O.beta_geometric(1000, 0.1, 3.0), O.dmax(p), 1)
    t0 = time.perf_counter()
    O.sample(p, thr, R, RUN_SEED0, start=0, phase=0, r0=r0)
    return time.perf_counter() - t0


def _oracle_solve_worker(start):
    """One Multi-start SPVAR start of the TTS99 workload, solved by the oracle."""
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_1706_07826_gb300 import instances as I
    inst = I.cubic3d(TTS_L, TTS_SEED)
    p = O.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J, inst.h)
    thr = O.thresholds(O.beta_geometric(TTS_T, 0.1, 3.0), O.dmax(p), 1)
    t0 = time.perf_counter()
    r = O.solve(p, thr, TTS_RUN_SEED, num_starts=1, start0=start, fixing_sample_size=TTS_S,
                solving_sample_size=TTS_S, elite_threshold=TTS_ELITE)
    return time.perf_counter() - t0, int(r.best_e[0])


def cpu_oracle_rate(replicas_per_core, cores=None, pool=None):
    """Oracle SA sample of the workload's first phase, replicas split across
    the host cores (one process each).  Returns (attempts/s, cores, seconds)."""
    cores = cores or os.cpu_count() or 1
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(cores)
        pool.map(_oracle_worker, [(0, 1)] * cores)  # start-up outside the timing
    try:
        t0 = time.perf_counter()
        pool.map(_oracle_worker, [(c * replicas_per_core, replicas_per_core) for c in range(cores)])
        dt = time.perf_counter() - t0
    finally:
        if own:
            pool.close()
            pool.join()
    attempts = cores * replicas_per_core * 512 * 1000
    return attempts / dt, cores, dt


def cpu_oracle_tts(pool, cores):
    """The oracle solving one TTS99 start per host core at once: wall time and
    each start's best energy."""
    t0 = time.perf_counter()
    res = pool.map(_oracle_solve_worker, list(range(cores)))
    return time.perf_counter() - t0, [b for _, b in res]


def reference_arm(args, rank, world):
    if rank != 0:
        return
    R = args.ref_replicas
    cores = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(cores)
    for _ in range(args.warmup):
        cpu_oracle_rate(1, cores, pool)
    vals, secs = [], 0.0
    for _ in range(args.steps):
        v, _, dt = cpu_oracle_rate(R, cores, pool)
        vals.append(v)
        secs += dt
    pool.close()
    pool.join()
    value = args.steps * cores * R * 512 * 1000 / secs
    cfg = dict(WORKLOAD)
    sample = ("oracle SA sample of the first phase of start 0: %d replicas x 512 spins x 1000 sweeps per step "
              "(%d per core, one process per core)" % (cores * R, R))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ GPU arm
class Peaks:
    """Measured integer issue ceilings of this GPU (thread-level ops/s)."""

    def __init__(self, spvar):
        self.rate = {}
        for form in range(6):
            self.rate[form], _ = spvar.measure_issue_rate(form, 20000)
        self.issue = self.rate[3]  # lop3 + mad.lo on alternate chains: both integer pipes busy
        self.wide = self.rate[4]

    def roof(self, attempts, sweep_ms, ops_per_attempt):
        """Roofline of a sweep kernel from its attempts and event-timed duration."""
        if not sweep_ms or sweep_ms <= 0:
            return None
        aps = attempts / (sweep_ms / 1000.0)
        achieved = aps * ops_per_attempt / 1e12
        wide_cap = self.wide / WIDE_PER_ATTEMPT
        return {"bound": "alu", "achieved": achieved, "peak": self.issue / 1e12, "unit": "Tops/s",
                "frac": achieved * 1e12 / self.issue, "ops_per_attempt": ops_per_attempt,
                "wide_mul_cap": wide_cap, "wide_frac": aps / wide_cap}

    def summary(self):
        from paper_1706_07826_gb300 import spvar
        return {spvar.ISSUE_FORMS[f]: self.rate[f] for f in range(6)}


def ops_per_attempt(inst, extra=0.0):
    return PHILOX_OPS_PER_ATTEMPT + 2.0 * inst.m / max(inst.n, 1) + ACCEPT_OPS_PER_ATTEMPT + extra


def run_form(spvar, torch, plan, K, W, seeds0, flush, profile=False, nvtx="c2"):
    """W warm-up + K timed plan runs; returns (total ms, attempts list, outs)."""
    stream = torch.cuda.current_stream()
    attempts = []
    for w in range(W):
        plan.run(seeds0 + w, device=True)
    torch.cuda.synchronize()
    plan.set_profiling(profile)
    sweep_ms, sweep_n = 0.0, 0
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    out = plan.alloc_outputs(True)
    best = []
    for k in range(K):
        flush.add_(1)
        torch.cuda.nvtx.range_push(nvtx)
        evs[k][0].record(stream)
        plan.run(seeds0 + 100 + k, out=out, device=True)
        evs[k][1].record(stream)
        torch.cuda.nvtx.range_pop()
        if profile:
            ms, n = plan.sweep_time()
            sweep_ms += ms
            sweep_n += n
        a, _ = plan.stats()
        attempts.append(a)
        best.append(out.best_energy.min().item())
    torch.cuda.synchronize()
    total = sum(a.elapsed_time(b) for a, b in evs)
    plan.set_profiling(False)
    return total, attempts, best, (sweep_ms, sweep_n), out


def profiled_traffic(kernel_kind):
    """DRAM bytes per launch of the sweep kernel from the committed ncu
    summary, or None when the kernel's source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "k_sweep_pm1_chimera_c8.md")
    if kernel_kind != "pm1-register" or not os.path.exists(path):
        return None
    text = open(path).read()
    vals = dict(l.split(": ", 1) for l in text.splitlines()
                if l.startswith(("dram_bytes_per_launch:", "kernel_source_sha256_16:")))
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return int(vals["dram_bytes_per_launch"])


def kernel_source_hash():
    """Hash of what the register sweep kernel is compiled from: its own sources
    and the device structs it reads (not the host-side parts of the header)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1706_07826_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("sweep_pm1.cu", "sweep_common.cuh", "philox.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    text = open(os.path.join(csrc, "spvar_internal.h")).read()
    for name in ("DevProb", "SweepJob", "WorkItem", "SweepLaunch"):
        start = text.index("struct %s {" % name)
        h.update(text[start:text.index("};", start) + 2].encode())
    return h.hexdigest()[:16]


def timed_plan(spvar, torch, plan, seeds, flush, name):
    """One untimed run, one timed run (CUDA events), one profiled run (sweep
    kernel time); returns (attempts/s, ms, attempts, sweep ms, launches, out)."""
    plan.run([s + 7919 for s in seeds], device=True)
    torch.cuda.synchronize()
    flush.add_(1)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push(name)
    a.record()
    out = plan.run(seeds, device=True)
    b.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    att, _ = plan.stats()
    plan.set_profiling(True)
    torch.cuda.nvtx.range_push(name + "_profiled")
    plan.run(seeds, device=True)
    torch.cuda.nvtx.range_pop()
    sweep_ms, sweep_n = plan.sweep_time()
    plan.set_profiling(False)
    return att / (ms / 1000.0), ms, att, sweep_ms, sweep_n, out


def measure_config(spvar, torch, flush, peaks, probs, insts, kw, seeds, name, plain=True):
    """Batched (and plain) form of one configuration with the batched sweep
    kernel's roofline."""
    res = {}
    for form, fname in ((spvar.FORM_BATCHED, "batched"), (spvar.FORM_PLAIN, "plain")):
        if fname == "plain" and not plain:
            continue
        plan = spvar.Plan(probs, spvar.make_params(form=form, **kw))
        aps, ms, att, sweep_ms, sweep_n, out = timed_plan(spvar, torch, plan, seeds, flush, name + "_" + fname)
        if fname == "batched":
            res["value"] = aps
            mean_deg_ops = sum(ops_per_attempt(x) * x.n for x in insts) / sum(x.n for x in insts)
            roof = peaks.roof(att, sweep_ms, mean_deg_ops)
            if roof:
                res["frac"] = roof["frac"]
                res["wide_frac"] = roof["wide_frac"]
            res["kernel"] = plan.shape()["kernel"]
        else:
            res["plain"] = aps
            res["speedup"] = res["value"] / aps
        plan.close()
    return res


def measure_c1_c3(spvar, torch, flush, peaks):
    """c1 (3D L=4, ISPVAR until every spin is fixed, 1 start, 256 samples,
    1000 sweeps) and c3 (weak-strong Chimera C12 x100, 32 starts, 250 + 250
    samples), batched and plain."""
    from paper_1706_07826_gb300 import instances as I
    out = {}
    c1 = I.cubic3d(4, 1100)
    r = measure_config(spvar, torch, flush, peaks, [spvar.Problem.from_instance(c1)], [c1],
                       dict(num_starts=1, fixing_sample_size=256, solving_sample_size=0, num_sweeps=1000,
                            elite_threshold=0.1, iterate=True, max_fix_phases=64), [2], "c1")
    out["c1"] = r
    c3 = I.weak_strong(12, 1300)
    r = measure_config(spvar, torch, flush, peaks, [spvar.Problem.from_instance(c3)], [c3],
                       dict(num_starts=32, fixing_sample_size=250, solving_sample_size=250, num_sweeps=1000,
                            elite_threshold=0.2), [2], "c3")
    out["c3"] = r
    return out


def measure_uneven(spvar, torch, flush, peaks):
    """c4: 64 3D +-J instances, L uniform in 6..12, 2000 + 2000 samples, 1000
    sweeps, one persistent launch per phase for all of them (batched) vs plain."""
    from paper_1706_07826_gb300 import instances as I
    insts = I.uneven_batch(64, 6, 12, seed=1400)
    probs = [spvar.Problem.from_instance(x) for x in insts]
    seeds = [1401 + i for i in range(len(insts))]
    return measure_config(spvar, torch, flush, peaks, probs, insts,
                          dict(num_starts=1, fixing_sample_size=2000, solving_sample_size=2000, num_sweeps=1000,
                               elite_threshold=0.1), seeds, "c4")


def measure_sweeps_per_launch(spvar, torch, flush, peaks):
    """The autotuner's sweeps-per-launch axis, measured on the headline
    workload: one sweep launch per phase against four (each resuming from the
    states the previous one wrote)."""
    inst = _instance()
    prob = spvar.Problem.from_instance(inst)
    out = {}
    for spl, name in ((1000, "one"), (250, "four")):
        prm = _params(spvar.FORM_BATCHED)
        prm.sweeps_per_launch = spl
        plan = spvar.Plan([prob], prm)
        aps, ms, att, sweep_ms, sweep_n, _ = timed_plan(spvar, torch, plan, [77], flush, "spl_" + name)
        out[name] = aps
        plan.close()
    return out


def measure_sqa(spvar, torch, flush, peaks):
    """Second sampler (SQA, discrete-time path integral): Multi-start SPVAR on
    Chimera C8 with SQA in every phase, 10 starts x (500 + 500) runs, 16 Trotter
    slices, 1000 sweeps, beta 3, transverse field 3 -> 0.01.  An attempt is one
    spin-slice update (two slice neighbours added to the local field)."""
    from paper_1706_07826_gb300 import instances as I
    inst = I.chimera(8, 1100)
    prob = spvar.Problem.from_instance(inst)
    prm = spvar.make_params(num_starts=10, fixing_sample_size=500, solving_sample_size=500, num_sweeps=1000,
                            elite_threshold=0.1, sampler=spvar.SAMPLER_SQA, sqa_slices=16, sqa_beta=3.0,
                            sqa_gamma0=3.0, sqa_gamma1=0.01)
    plan = spvar.Plan([prob], prm)
    aps, ms, att, sweep_ms, sweep_n, out = timed_plan(spvar, torch, plan, [2300], flush, "sqa_c8")
    plan.close()
    roof = peaks.roof(att, sweep_ms, ops_per_attempt(inst, 2.0))
    return {"value": aps, "frac": roof["frac"] if roof else None, "best": int(out.best_energy.min().item())}


def measure_pticm(spvar, torch, flush):
    """PTICM (Sec. III.D) on a 3D +-J L=10 problem: 304 independent runs, 32
    inverse temperatures geometric 0.2 -> 3.0, two replicas each, cluster
    moves and kept lists (K = 10) in the lower half, 1000 sweeps."""
    from paper_1706_07826_gb300 import instances as I
    inst = I.cubic3d(10, 1600)
    prob = spvar.Problem.from_instance(inst)
    betas = np.geomspace(0.2, 3.0, 32)
    T, runs = 1000, 304
    dx = spvar.energy_range(inst)
    torch.cuda.nvtx.range_push("pticm_3d_L10_short")  # the warm-up launch, 20 sweeps: the case profiles capture
    spvar.pticm_sample(prob, betas, 20, dx, K=10, num_runs=runs, seed=3)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    flush.add_(1)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("pticm_3d_L10")
    a.record()
    out = spvar.pticm_sample(prob, betas, T, dx, K=10, num_runs=runs, seed=4)
    b.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    att = runs * 2 * len(betas) * inst.n * T
    return {"value": att / (ms / 1000.0), "best": int(out["kept_e"][:, :, 0].min().item())}


def measure_pticm_spvar(spvar, torch, flush):
    """Alg. 2 with PTICM as the sampler of every phase (Sec. III.D sample) on 3D
    +-J L=10: 304 starts (two runs per SM), 16 temperatures geometric 0.2 -> 3.0,
    10 kept states per tracked replica (160-state samples), 1000 sweeps, elite
    0.2; attempts count every replica's Metropolis proposals."""
    from paper_1706_07826_gb300 import instances as I
    inst = I.cubic3d(10, 1600)
    prob = spvar.Problem.from_instance(inst)
    S = spvar.pticm_sample_size(16, 10)
    prm = spvar.make_params(num_starts=304, fixing_sample_size=S, solving_sample_size=S, num_sweeps=1000,
                            elite_threshold=0.2, sampler=spvar.SAMPLER_PTICM, pticm_temps=16, pticm_keep=10,
                            pticm_beta0=0.2, pticm_beta1=3.0)
    plan = spvar.Plan([prob], prm)
    aps, ms, att, sweep_ms, sweep_n, out = timed_plan(spvar, torch, plan, [1601], flush, "pticm_spvar")
    nfree = out.nfree.cpu().numpy()
    plan.close()
    return {"value": aps, "ms": ms, "best": int(out.best_energy.min().item()),
            "fixed_frac": float(1.0 - nfree[:, 1].mean() / inst.n)}


def _hbm_peak_gbs():
    """Measured copy bandwidth of this GPU pool (GB/s), or the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measure_persistence_scaled(spvar, torch):
    """The persistence pass (elite, counts and fixing, fold and compact) at a
    scale where HBM matters: 64 3D +-J problems of N = 8000 in one plan, 2000
    samples per phase, one launch per kernel for all of them.  Algorithmic
    bytes per problem: energies 8S, elite rows k ceil(N/32) 4, counts and fixes
    5N, the CSR and layout read (4(N+1) + 8 nnz + 13N) and the reduced one
    written (28N' + 12 nnz'), and the solving phase's energies 8S."""
    from paper_1706_07826_gb300 import instances as I
    insts = [I.cubic3d(20, 1700 + i) for i in range(64)]
    probs = [spvar.Problem.from_instance(x) for x in insts]
    S, T = 2000, 20
    prm = spvar.make_params(num_starts=1, fixing_sample_size=S, solving_sample_size=S, num_sweeps=T,
                            elite_threshold=0.1)
    plan = spvar.Plan(probs, prm)
    seeds = [1800 + i for i in range(64)]
    plan.run(seeds, device=True)
    torch.cuda.synchronize()
    plan.set_profiling(True)
    out = plan.run([x + 1 for x in seeds], device=False)
    post_ms = plan.post_time()
    plan.close()
    k = int(np.ceil(0.1 * S))
    total = 0
    off = 0
    for i, x in enumerate(insts):
        n, nnz = x.n, 2 * x.m
        fixed = np.asarray(out.fixed[off:off + n])
        off += n
        free = fixed == 0
        n2 = int(free.sum())
        nnz2 = 2 * int(np.sum(free[x.ei] & free[x.ej]))
        total += 8 * S + k * ((n + 31) // 32) * 4 + 5 * n
        total += 4 * (n + 1) + 8 * nnz + 13 * n + 28 * n2 + 12 * nnz2
        total += 8 * S
    peak, kind = _hbm_peak_gbs()
    gbs = total / (post_ms / 1000.0) / 1e9
    return {"gbs": gbs, "frac": gbs / peak, "peak": kind, "bytes": total, "ms": post_ms}


def measure_serving(spvar, peaks, count=12):
    """c5: Poisson arrivals of 3D +-J instances, L in 8..20, through the
    continuous-batching server (background engine, 500-sweep steps): p50/p99
    latency, attempts/s and the sweep kernel's roofline.  The arrival rate is
    0.7 x the capacity measured on two saturating requests."""
    from paper_1706_07826_gb300 import instances as I
    prm = spvar.make_params(num_starts=20, fixing_sample_size=250, solving_sample_size=250, num_sweeps=5000,
                            elite_threshold=0.2, sweep_kernel=spvar.SWEEP_PM1)
    srv = spvar.Server(prm, 8 << 30, max_n=8000, max_nnz=48000, max_degree=6, max_dmax=12, max_requests=32,
                       sweeps_per_step=500)
    srv.start()
    cal = [I.cubic3d(14, 1590 + i) for i in range(2)]
    t0 = time.perf_counter()
    ids = [srv.submit(x, 1) for x in cal]
    infos = [srv.info(i, timeout=600.0) for i in ids]
    dt = time.perf_counter() - t0
    cap_attempts = sum(i.attempts for i in infos) / dt
    mean_att = 20 * 500 * 5000 * np.mean([L ** 3 for L in range(8, 21)])
    rate = 0.7 * cap_attempts / mean_att
    arrivals, insts = I.poisson_stream(count, rate, 8, 20, seed=1500)
    ms0, _ = srv.sweep_time()
    t0 = time.perf_counter()
    ids = []
    for ta, inst in zip(arrivals, insts):
        wait = t0 + ta - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        ids.append(srv.submit(inst, 1501 + len(ids)))
    infos = [srv.info(i, timeout=1200.0) for i in ids]
    t_end = time.perf_counter()
    srv.stop()
    ms1, _ = srv.sweep_time()
    lat = np.array([i.latency_s for i in infos])
    att = sum(i.attempts for i in infos)
    srv.close()
    ops = sum(ops_per_attempt(x) * x.n for x in insts) / sum(x.n for x in insts)
    roof = peaks.roof(att, ms1 - ms0, ops)
    return {"value": att / (t_end - t0), "capacity": cap_attempts, "rate": rate,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "frac": roof["frac"] if roof else None}


def measure_tts99(spvar, torch, flush, peaks, oracle_tts):
    """TTS99 (Sec. III.A: R99 in wall time) on 3D +-J L = 12 (N = 1728) at
    1000 sweeps, 200 starts x (250 + 250) samples, elite 0.2, where the
    per-start success rate is strictly between 0 and 1.  E_known = the lowest
    energy of independent long runs (PTICM, 152 runs at 10^4 sweeps; SA, 4000
    samples at 2 x 10^4 sweeps): best known, not proved.  SA alone draws 500
    samples per start (the same sample budget).  Each form's p comes from its
    own starts (plain: other seeds)."""
    from paper_1706_07826_gb300 import instances as I
    from paper_1706_07826_gb300 import metrics as MT
    inst = I.cubic3d(TTS_L, TTS_SEED)
    prob = spvar.Problem.from_instance(inst)
    dmax = prob.info().dmax
    # independent best-known energy
    pt = spvar.pticm_sample(prob, np.geomspace(0.2, 3.0, 32), 10000, spvar.energy_range(inst), K=10, num_runs=152,
                            seed=77)
    thr_l = spvar.thresholds(spvar.beta_geometric(20000, 0.1, 3.0), dmax, 1)
    _, e_l = spvar.sample(prob, spvar.thresholds_device(thr_l), thr_l.shape[1], 20000, 4000, 99, 0, 0)
    torch.cuda.synchronize()
    e_known = min(int(pt["kept_e"][:, :, 0].min().item()), int(e_l.min().item()))
    out = {"e_known": e_known}
    att_start = 2 * TTS_S * TTS_T * inst.n  # upper bound: the solving phase anneals the reduced problem
    # SA alone: 500 samples per start
    thr = spvar.thresholds(spvar.beta_geometric(TTS_T, 0.1, 3.0), dmax, 1)
    thr_d = spvar.thresholds_device(thr)
    spvar.sample(prob, thr_d, thr.shape[1], TTS_T, 2 * TTS_S, 5, 0, 0)
    torch.cuda.synchronize()
    flush.add_(1)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    es = [spvar.sample(prob, thr_d, thr.shape[1], TTS_T, 2 * TTS_S, TTS_RUN_SEED, st, 0)[1]
          for st in range(TTS_STARTS)]
    b.record()
    torch.cuda.synchronize()
    best_sa = [int(e.min().item()) for e in es]
    p = MT.fraction_solved(best_sa, e_known)
    s99 = MT.starts99(p)
    sec = a.elapsed_time(b) / 1000.0 / TTS_STARTS
    out["sa"] = {"p": p, "s": s99 * sec if s99 else None}
    best_b = None
    for form, name, seed in ((spvar.FORM_BATCHED, "batched", TTS_RUN_SEED), (spvar.FORM_PLAIN, "plain",
                                                                              TTS_RUN_SEED + 1)):
        plan = spvar.Plan([prob], spvar.make_params(num_starts=TTS_STARTS, fixing_sample_size=TTS_S,
                                                    solving_sample_size=TTS_S, num_sweeps=TTS_T,
                                                    elite_threshold=TTS_ELITE, form=form))
        aps, ms, att, sweep_ms, sweep_n, o = timed_plan(spvar, torch, plan, [seed], flush, "tts_" + name)
        plan.close()
        best = o.best_energy.cpu().numpy()
        p = MT.fraction_solved(best, e_known)
        s99 = MT.starts99(p)
        sec = ms / 1000.0 / TTS_STARTS
        out[name] = {"p": p, "s": s99 * sec if s99 else None}
        if name == "batched":
            best_b = best
            att_start = att / TTS_STARTS
            p_b = p
            if s99:
                # the same starts at the measured issue ceiling (sweep only)
                out["roof_s"] = s99 * att_start * ops_per_attempt(inst) / peaks.issue
                out["roof_frac"] = out["roof_s"] / out[name]["s"]
    if oracle_tts:
        wall, best_o = oracle_tts
        n = len(best_o)
        s99 = MT.starts99(p_b)
        # the oracle computes exactly what the GPU does: its starts' results equal the batched run's
        out["oracle"] = {"s": s99 * wall / n if s99 else None, "cores": n,
                         "same_as_gpu": bool(np.array_equal(np.asarray(best_o), best_b[:n]))}
    return out


def gpu_arm(args, rank, world):
    import torch
    from paper_1706_07826_gb300 import build as B
    from paper_1706_07826_gb300 import spvar
    if args.build:
        B.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))

    cpu, oracle_tts = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # before any GPU work: spawned oracle processes on the host cores
        R = args.cpu_replicas
        cores = os.cpu_count() or 1
        pool = mp.get_context("spawn").Pool(cores)
        pool.map(_oracle_worker, [(0, 1)] * cores)
        rate, cores, dt = cpu_oracle_rate(R, cores, pool)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "headline phase 0: %d replicas x 512 spins x 1000 sweeps, %d per core, %.1f s"
                         % (cores * R, R, dt)}
        if not args.no_extra:
            oracle_tts = cpu_oracle_tts(pool, cores)
        pool.close()
        pool.join()

    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))

    inst = _instance()
    seed_base = RUN_SEED0
    prob = spvar.Problem.from_instance(inst)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    K, W = args.steps, args.warmup

    with ClockSampler(dev) as clk_peak:
        peaks = Peaks(spvar)
    plan_b = spvar.Plan([prob], _params(spvar.FORM_BATCHED, rank))
    plan_p = spvar.Plan([prob], _params(spvar.FORM_PLAIN, rank))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    with ClockSampler(dev) as clk:
        tb, att_b, best_b, _, out_b = run_form(spvar, torch, plan_b, K, W, seed_base, flush, nvtx="c2_batched")
    barrier()
    # profiled pass: same runs, sweep kernel timed with events on the launch stream
    Kp = max(3, K // 5)
    _, att_prof, _, (sweep_ms, sweep_n), _ = run_form(spvar, torch, plan_b, Kp, 1, seed_base, flush, profile=True,
                                                       nvtx="c2_batched_profiled")
    tp, att_p, best_p, _, out_p = run_form(spvar, torch, plan_p, Kp, 1, seed_base, flush, nvtx="c2_plain")
    barrier()

    t_b = torch.tensor([tb], dtype=torch.float64, device="cuda")
    n_b = torch.tensor([float(sum(att_b))], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t_b, op=dist.ReduceOp.MAX)
        dist.all_reduce(n_b, op=dist.ReduceOp.SUM)
    value = n_b.item() / (t_b.item() / 1000.0)
    plain_value = sum(att_p) / (tp / 1000.0)
    if dist:
        from paper_1706_07826_gb300 import distributed as D
        D.combine_best(out_b.best_energy.cpu().numpy(), device=torch.device("cuda", dev))

    # e2e through the public API with host buffers
    rp, col, val = spvar.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J)
    prm = _params(spvar.FORM_BATCHED, rank)
    h2d = rp.nbytes + col.nbytes + val.nbytes + inst.h.nbytes + 1000 * 13 * 4
    e2e_times, e2e_att = [], []
    for k in range(Kp + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pr = spvar.Problem.create(inst.n, rp, col, val, inst.h)
        o = spvar.solve(pr, prm, seed_base + 500 + k, device=False)
        dt = time.perf_counter() - t0
        if k > 0:
            e2e_times.append(dt)
            e2e_att.append(int((o.counts.astype(np.int64) * o.nfree).sum()) * 1000)
        pr.close()
    d2h = sum(getattr(o, f).nbytes for f in ("energies", "counts", "nfree", "nphases", "fixed", "best_energy",
                                             "best_state"))
    e2e_value = sum(e2e_att) / sum(e2e_times) * world

    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        extra["tts99"] = measure_tts99(spvar, torch, flush, peaks, oracle_tts)
        extra.update(measure_c1_c3(spvar, torch, flush, peaks))
        extra["c4"] = measure_uneven(spvar, torch, flush, peaks)
        extra["c5"] = measure_serving(spvar, peaks)
        extra["sqa"] = measure_sqa(spvar, torch, flush, peaks)
        extra["pticm"] = measure_pticm(spvar, torch, flush)
        extra["pticm_spvar"] = measure_pticm_spvar(spvar, torch, flush)
        extra["persist"] = measure_persistence_scaled(spvar, torch)
        extra["spl"] = measure_sweeps_per_launch(spvar, torch, flush, peaks)

    # roofline of the headline sweep kernel (integer issue bound)
    opa = ops_per_attempt(inst)
    att_per_launch = sum(att_prof) / max(sweep_n, 1)
    ms_per_launch = sweep_ms / max(sweep_n, 1)
    roof = peaks.roof(att_per_launch, ms_per_launch, opa)
    shape = plan_b.shape()
    cs = clk.summary()
    if cpu:
        cpu["per_core"] = cpu["value"] / cpu["cores"]
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": tb / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": dict(WORKLOAD, form="batched", l2="256 MB written between steps",
                       parallelism="starts sharded per rank" if world > 1 else "single GPU", sweep_shape=shape),
        "roofline": dict(roof, traffic=profiled_traffic(shape["kernel"]), kernel="k_sweep_pm1",
                         ms_per_launch=ms_per_launch, peak_kind="measured issue probe"),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "api": "problem_create+solve", "ms_per_step": 1000 * statistics.mean(e2e_times)},
        # per run: slot init, then per sweep launch of each of the two phases the work list, the
        # sweep, the persistence pass (one cluster per start) and the loop-condition kernel
        "gpu_launches": K * (1 + 2 * -(-1000 // max(shape["sweeps_per_launch"], 1)) * 4),
        "clocks": cs,
        "plain": {"value": plain_value, "speedup": value / world / plain_value},
        "peaks": dict(peaks.summary(), sm_mhz=clk_peak.summary()["sm_mhz"]),
    }
    line.update(extra)
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(r4(line), separators=(",", ":")), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-replicas", type=int, default=400, help="oracle replicas per core (cpu_baseline)")
    ap.add_argument("--ref-replicas", type=int, default=24, help="oracle replicas per core per step (reference arm)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-build", dest="build", action="store_false")
    ap.add_argument("--no-extra", action="store_true", help="only the headline workload")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
    else:
        gpu_arm(args, rank, world)


if __name__ == "__main__":
    main()
