"""Thin ctypes binding of ``libspvar.so`` (declared in ``include/spvar.h``).

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch supplies device memory (tensors) and streams; numpy arrays carry host
inputs.  The library must have been built (``__graft_entry__.build()`` or
``python -m paper_1706_07826_gb300.build``); there is no fallback of any kind.
"""
import ctypes
import dataclasses
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspvar.so")

OK, EINVAL, EOVERFLOW, ENOMEM, EBUDGET, ETIMEOUT, ECUDA, ELIMIT = 0, -1, -2, -3, -4, -5, -6, -7
FORM_BATCHED, FORM_PLAIN = 0, 1
SWEEP_AUTO, SWEEP_GENERAL, SWEEP_PM1, SWEEP_PM1S, SWEEP_PM1W, SWEEP_PM1Q = 0, 1, 2, 3, 4, 5
SAMPLER_SA, SAMPLER_SQA, SAMPLER_PTICM = 0, 1, 2
MAX_N, MAX_DEGREE, MAX_SWEEPS, MAX_PHASE, MAX_SAMPLES = 32768, 32, 1048574, 4095, 16384
NOALLOC_MAX_N = 16384

vp = ctypes.c_void_p
i32 = ctypes.c_int32
i64 = ctypes.c_int64
u32 = ctypes.c_uint32
u64 = ctypes.c_uint64


class SpvarError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (what, _strerror(code), code))


class ProblemInfo(ctypes.Structure):
    _fields_ = [("n", i32), ("nnz", i32), ("ncol", i32), ("maxdeg", i32), ("dmax", i32),
                ("hzero", i32), ("pm1", i32), ("energy_scale", i32), ("offset", i64)]


class Params(ctypes.Structure):
    _fields_ = [("num_starts", i32), ("fixing_sample_size", i32), ("solving_sample_size", i32),
                ("num_sweeps", i32), ("beta0", ctypes.c_double), ("beta1", ctypes.c_double),
                ("elite_threshold", ctypes.c_double), ("fix_num", i32), ("fix_den", i32),
                ("iterate", i32), ("max_fix_phases", i32), ("canon", i32), ("form", i32),
                ("replicas_per_block", i32), ("sweep_kernel", i32), ("sweep_block", i32), ("start_offset", i32),
                ("component_boost", i32), ("tree_preprocess", i32), ("corr_sample_size", i32),
                ("corr_num", i32), ("corr_den", i32), ("corr_elite_threshold", ctypes.c_double),
                ("sampler", i32), ("sqa_slices", i32), ("sqa_beta", ctypes.c_double), ("sqa_gamma0", ctypes.c_double),
                ("sqa_gamma1", ctypes.c_double), ("sweeps_per_launch", i32), ("pticm_temps", i32),
                ("pticm_keep", i32), ("pticm_beta0", ctypes.c_double), ("pticm_beta1", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("params", Params), ("budget_bytes", ctypes.c_size_t), ("max_n", i32), ("max_nnz", i32),
                ("max_degree", i32), ("max_dmax", i32), ("energy_scale", i32), ("max_requests", i32),
                ("sweeps_per_step", i32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", i32), ("n", i32), ("best_energy", i64), ("latency_s", ctypes.c_double),
                ("queue_s", ctypes.c_double), ("attempts", i64)]


class Result(ctypes.Structure):
    _fields_ = [("device", i32), ("energies", vp), ("counts", vp), ("nfree", vp), ("nphases", vp),
                ("fixed", vp), ("best_energy", vp), ("best_state", vp)]


_lib = None


def lib():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libspvar.so is missing (%s): build it with __graft_entry__.build(); "
                               "there is no CPU fallback" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        L.spvar_strerror.restype = ctypes.c_char_p
        L.spvar_strerror.argtypes = [ctypes.c_int]
        L.spvar_device_count.argtypes = [ctypes.POINTER(ctypes.c_int)]
        L.spvar_csr_from_edges.argtypes = [i32, i64, vp, vp, vp, vp, vp, vp]
        L.spvar_problem_create.argtypes = [i32, vp, vp, vp, vp, i64, i32, vp, ctypes.POINTER(vp)]
        L.spvar_problem_destroy.argtypes = [vp]
        L.spvar_problem_destroy.restype = None
        L.spvar_problem_get_info.argtypes = [vp, ctypes.POINTER(ProblemInfo)]
        L.spvar_problem_download.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.spvar_beta_geometric.argtypes = [i32, ctypes.c_double, ctypes.c_double, vp]
        L.spvar_thresholds.argtypes = [i32, vp, i32, i32, vp]
        L.spvar_sample.argtypes = [vp, i32, vp, i32, i32, u64, u32, u32, vp, vp, vp]
        L.spvar_sqa_table.argtypes = [i32, i32, vp, vp, i32, i32, vp]
        L.spvar_gamma_linear.argtypes = [i32, ctypes.c_double, ctypes.c_double, vp]
        L.spvar_sqa_sample.argtypes = [vp, i32, i32, vp, i32, i32, u64, u32, u32, vp, vp, vp, vp]
        L.spvar_pticm_sample.argtypes = [vp, i32, i32, vp, i32, vp, i32, i32, i32, i32, i32, i32, u64, u32, u32,
                                         vp, vp, vp, vp, vp, vp]
        L.spvar_sample_range.argtypes = [vp, i32, i32, vp, i32, i32, u64, u32, u32, vp, vp, vp, vp]
        L.spvar_persistence.argtypes = [vp, i32, vp, vp, ctypes.c_double, i32, i32, i32, vp, vp, vp, vp,
                                        ctypes.POINTER(i32), vp]
        L.spvar_reduce.argtypes = [vp, vp, vp, vp, ctypes.POINTER(vp)]
        L.spvar_reduce_noalloc.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.spvar_plan_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(Params), ctypes.c_size_t, vp,
                                        ctypes.POINTER(vp)]
        L.spvar_plan_workspace_bytes.argtypes = [vp]
        L.spvar_plan_workspace_bytes.restype = ctypes.c_size_t
        L.spvar_plan_run.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(Result), vp]
        L.spvar_plan_destroy.argtypes = [vp]
        L.spvar_plan_destroy.restype = None
        L.spvar_plan_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32)]
        L.spvar_plan_sweeps_per_launch.argtypes = [vp, ctypes.POINTER(i32)]
        L.spvar_solve.argtypes = [vp, ctypes.POINTER(Params), u64, ctypes.POINTER(Result), vp]
        L.spvar_solve_cache_release.argtypes = []
        L.spvar_solve_cache_release.restype = None
        L.spvar_plan_set_profiling.argtypes = [vp, i32]
        L.spvar_plan_sweep_time.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
        L.spvar_plan_shape.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                       ctypes.POINTER(i32)]
        L.spvar_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
        L.spvar_server_submit.argtypes = [vp, i32, vp, vp, vp, vp, i64, u64, ctypes.POINTER(i64)]
        L.spvar_server_step.argtypes = [vp, ctypes.POINTER(i32)]
        L.spvar_server_start.argtypes = [vp]
        L.spvar_server_stop.argtypes = [vp]
        L.spvar_server_wait.argtypes = [vp, i64, ctypes.c_double, ctypes.POINTER(RequestInfo)]
        L.spvar_server_result.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
        L.spvar_server_release.argtypes = [vp, i64]
        L.spvar_server_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                         ctypes.POINTER(i32)]
        L.spvar_measure_issue_rate.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double), vp]
        L.spvar_server_sweep_time.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
        L.spvar_server_destroy.argtypes = [vp]
        L.spvar_server_destroy.restype = None
        _lib = L
    return _lib


def _strerror(code):
    try:
        return lib().spvar_strerror(code).decode()
    except Exception:  # library not loadable: still report the code
        return "error"


def _check(rc, what):
    if rc != OK:
        raise SpvarError(rc, what)


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _hp(a):
    return a.ctypes.data_as(vp) if a is not None and a.size else None


def _dp(t):
    """Device pointer of a CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return vp(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return vp(s.cuda_stream)


def device_count():
    c = ctypes.c_int(0)
    _check(lib().spvar_device_count(ctypes.byref(c)), "spvar_device_count")
    return c.value


# --------------------------------------------------------------- problem
def csr_from_edges(n, ei, ej, J):
    """Edge list -> symmetric CSR (host); each pair once, i != j."""
    ei, ej, J = _host(ei, np.int32), _host(ej, np.int32), _host(J, np.int32)
    m = len(ei)
    rp = np.zeros(n + 1, np.int32)
    col = np.zeros(max(2 * m, 1), np.int32)
    val = np.zeros(max(2 * m, 1), np.int32)
    _check(lib().spvar_csr_from_edges(n, m, _hp(ei), _hp(ej), _hp(J), _hp(rp), _hp(col), _hp(val)),
           "spvar_csr_from_edges")
    return rp, col[:2 * m].copy(), val[:2 * m].copy()


class Problem:
    """Owning handle of a device-resident problem (Sec. I)."""

    def __init__(self, handle):
        self.handle = handle

    @classmethod
    def create(cls, n, row_ptr, col, val, h, offset=0, scale=1, stream=None):
        rp, c, v, hh = (_host(row_ptr, np.int32), _host(col, np.int32), _host(val, np.int32),
                        _host(h, np.int32))
        out = vp()
        _check(lib().spvar_problem_create(n, _hp(rp), _hp(c), _hp(v), _hp(hh), int(offset), int(scale),
                                          _stream(stream), ctypes.byref(out)), "spvar_problem_create")
        return cls(out)

    @classmethod
    def from_instance(cls, inst, stream=None):
        rp, c, v = csr_from_edges(inst.n, inst.ei, inst.ej, inst.J)
        return cls.create(inst.n, rp, c, v, inst.h, inst.offset, inst.scale, stream)

    def info(self):
        i = ProblemInfo()
        _check(lib().spvar_problem_get_info(self.handle, ctypes.byref(i)), "spvar_problem_get_info")
        return i

    @property
    def n(self):
        return self.info().n

    def download(self, stream=None):
        i = self.info()
        rp = np.zeros(i.n + 1, np.int32)
        col = np.zeros(max(i.nnz, 1), np.int32)
        val = np.zeros(max(i.nnz, 1), np.int32)
        h = np.zeros(max(i.n, 1), np.int32)
        colour = np.zeros(max(i.n, 1), np.int32)
        _check(lib().spvar_problem_download(self.handle, _hp(rp), _hp(col), _hp(val), _hp(h), _hp(colour),
                                            _stream(stream)), "spvar_problem_download")
        return dict(n=i.n, row_ptr=rp, col=col[:i.nnz], val=val[:i.nnz], h=h[:i.n], colour=colour[:i.n],
                    offset=i.offset, ncol=i.ncol, dmax=i.dmax, hzero=i.hzero, pm1=i.pm1)

    def close(self):
        if self.handle:
            lib().spvar_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------------- schedule
def beta_geometric(T, beta0, beta1):
    b = np.zeros(max(T, 1), np.float64)
    _check(lib().spvar_beta_geometric(T, beta0, beta1, _hp(b)), "spvar_beta_geometric")
    return b[:T]


def thresholds(beta, dmax, scale=1):
    beta = _host(beta, np.float64)
    thr = np.zeros((len(beta), dmax + 1), np.uint32)
    _check(lib().spvar_thresholds(len(beta), _hp(beta), dmax, scale, _hp(thr)), "spvar_thresholds")
    return thr


def thresholds_device(thr):
    """Host uint32 table -> CUDA int32 tensor holding the same bits."""
    import torch
    return torch.from_numpy(_host(thr, np.uint32).view(np.int32)).cuda()


def sqa_table(T, P, beta, gamma, dmax, scale=1):
    """Host acceptance entries of the SQA sweep, uint64 [T, 3, 2 (dmax/2) + 1];
    beta and gamma per sweep (or constants)."""
    beta = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, np.float64), (max(T, 1),)))
    gamma = np.ascontiguousarray(np.broadcast_to(np.asarray(gamma, np.float64), (max(T, 1),)))
    W = 2 * (dmax // 2) + 1
    ent = np.zeros((max(T, 1), 3, max(W, 1)), np.uint64)
    _check(lib().spvar_sqa_table(T, P, _hp(beta), _hp(gamma), dmax, scale, _hp(ent)), "spvar_sqa_table")
    return ent[:T]


def gamma_linear(T, gamma0, gamma1):
    """Transverse field falling linearly from gamma0 to gamma1 (endpoints included)."""
    g = np.zeros(max(T, 1), np.float64)
    _check(lib().spvar_gamma_linear(T, float(gamma0), float(gamma1), _hp(g)), "spvar_gamma_linear")
    return g[:T]


def table_device(ent):
    """Host uint64 SQA table -> CUDA int64 tensor holding the same bits."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(ent, np.uint64).view(np.int64)).cuda()


# ------------------------------------------------------------------ calls
def sample(problem, thr_dev, thr_stride, num_sweeps, num_samples, seed, start=0, phase=0,
           spins=None, energies=None, stream=None):
    """SA sample (Alg. 1 "obtain sample").  Returns (spins int32 [S, W], energies int64 [S])."""
    import torch
    n = problem.n
    W = (n + 31) // 32
    if spins is None:
        spins = torch.empty((max(num_samples, 1), max(W, 1)), dtype=torch.int32, device="cuda")
    if energies is None:
        energies = torch.empty(max(num_samples, 1), dtype=torch.int64, device="cuda")
    _check(lib().spvar_sample(problem.handle, num_sweeps, _dp(thr_dev), thr_stride, num_samples, seed, start,
                              phase, _dp(spins), _dp(energies), _stream(stream)), "spvar_sample")
    return spins, energies


def sqa_sample(problem, ent_dev, W, num_sweeps, P, num_samples, seed, start=0, phase=0, stream=None):
    """SQA sample (second sampler for Alg. 1): each run's lowest-energy Trotter slice.
    Returns (spins int32 [S, W], energies int64 [S], slice int32 [S])."""
    import torch
    n = problem.n
    Wn = (n + 31) // 32
    spins = torch.empty((max(num_samples, 1), max(Wn, 1)), dtype=torch.int32, device="cuda")
    energies = torch.empty(max(num_samples, 1), dtype=torch.int64, device="cuda")
    sl = torch.empty(max(num_samples, 1), dtype=torch.int32, device="cuda")
    _check(lib().spvar_sqa_sample(problem.handle, num_sweeps, P, _dp(ent_dev), W, num_samples, seed, start, phase,
                                  _dp(spins), _dp(energies), _dp(sl), _stream(stream)), "spvar_sqa_sample")
    return spins, energies, sl


def energy_range(inst):
    """An upper bound of max E - min E of an instance: 2 (sum |J| + sum |h|)."""
    return int(2 * (np.abs(np.asarray(inst.J, np.int64)).sum() + np.abs(np.asarray(inst.h, np.int64)).sum()))


def pticm_sample(problem, betas, num_sweeps, dx, K=10, num_runs=1, seed=0, start0=0, phase=0, icm_from=None,
                 keep_from=None, exchange=True, icm=True, stream=None):
    """PTICM runs (third sampler for Alg. 1, Sec. III.D): R = len(betas)
    ascending inverse temperatures, two replicas each; the sample of a run is
    the K lowest distinct states seen at each replica of temperatures
    >= keep_from (default R / 2).  dx >= max E - min E (energy_range).
    Returns dict of device tensors: kept int32 [runs, ntr, K, W], kept_e,
    nkept, final_states int32 [runs, 2R, W], final_e."""
    import torch
    betas = _host(betas, np.float64)
    R = len(betas)
    icm_from = R // 2 if icm_from is None else icm_from
    keep_from = R // 2 if keep_from is None else keep_from
    info = problem.info()
    dm, scale = info.dmax, info.energy_scale
    thr = thresholds_device(thresholds(betas, dm, scale))
    xthr = thresholds_device(thresholds(np.diff(betas) if R > 1 else np.zeros(1), dx, scale))
    n = problem.n
    Wn = max((n + 31) // 32, 1)
    ntr = 2 * (R - keep_from)
    runs1 = max(num_runs, 1)
    kept = torch.zeros((runs1, max(ntr, 1), K, Wn), dtype=torch.int32, device="cuda")
    kept_e = torch.zeros((runs1, max(ntr, 1), K), dtype=torch.int64, device="cuda")
    nkept = torch.zeros((runs1, max(ntr, 1)), dtype=torch.int32, device="cuda")
    final = torch.zeros((runs1, 2 * R, Wn), dtype=torch.int32, device="cuda")
    final_e = torch.zeros((runs1, 2 * R), dtype=torch.int64, device="cuda")
    flags = (1 if exchange else 0) | (2 if icm else 0)
    _check(lib().spvar_pticm_sample(problem.handle, R, num_sweeps, _dp(thr), dm + 1, _dp(xthr), dx, icm_from,
                                    keep_from, K, flags, num_runs, seed, start0, phase, _dp(kept), _dp(kept_e),
                                    _dp(nkept), _dp(final), _dp(final_e), _stream(stream)), "spvar_pticm_sample")
    return dict(kept=kept[:, :ntr], kept_e=kept_e[:, :ntr], nkept=nkept[:, :ntr], final_states=final,
                final_e=final_e)


def sample_range(problem, thr_dev, thr_stride, sweep_begin, sweep_end, num_samples, seed, start=0, phase=0,
                 init=None, spins=None, energies=None, stream=None):
    """Sweeps [sweep_begin, sweep_end) of a sample, continuing from `init`
    (bit-packed states of an earlier range; None only for sweep_begin = 0)."""
    import torch
    n = problem.n
    W = (n + 31) // 32
    if spins is None:
        spins = torch.empty((max(num_samples, 1), max(W, 1)), dtype=torch.int32, device="cuda")
    if energies is None:
        energies = torch.empty(max(num_samples, 1), dtype=torch.int64, device="cuda")
    _check(lib().spvar_sample_range(problem.handle, sweep_begin, sweep_end, _dp(thr_dev), thr_stride, num_samples,
                                    seed, start, phase, _dp(init), _dp(spins), _dp(energies), _stream(stream)),
           "spvar_sample_range")
    return spins, energies


def persistence(problem, num_samples, spins, energies, elite_threshold, fix_num=1, fix_den=1, canon=-1,
                stream=None):
    """Alg. 1 persistence.  Returns (elite [k], counts [n], fixed int8 [n], nfixed [1], k)."""
    import torch
    n = problem.n
    elite = torch.empty(max(num_samples, 1), dtype=torch.int32, device="cuda")
    counts = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    fixed = torch.empty(max(n, 1), dtype=torch.int8, device="cuda")
    nfixed = torch.empty(1, dtype=torch.int32, device="cuda")
    k = i32(0)
    _check(lib().spvar_persistence(problem.handle, num_samples, _dp(spins), _dp(energies), float(elite_threshold),
                                   fix_num, fix_den, canon, _dp(elite), _dp(counts), _dp(fixed), _dp(nfixed),
                                   ctypes.byref(k), _stream(stream)), "spvar_persistence")
    return elite[:k.value], counts[:n], fixed[:n], nfixed, k.value


def reduce(problem, fixed, stream=None):
    """Alg. 1 update of J and h.  Returns (reduced Problem, old_of_new int32 [n'])."""
    import torch
    n = problem.n
    old_of_new = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    out = vp()
    _check(lib().spvar_reduce(problem.handle, _dp(fixed), _dp(old_of_new), _stream(stream), ctypes.byref(out)),
           "spvar_reduce")
    red = Problem(out)
    return red, old_of_new[:red.n]


def reduce_noalloc(problem, fixed, row_ptr, col, val, h, offset, old_of_new, n_out, stream=None):
    """Allocation-free reduction into caller tensors (see spvar_reduce_noalloc)."""
    _check(lib().spvar_reduce_noalloc(problem.handle, _dp(fixed), _dp(row_ptr), _dp(col), _dp(val), _dp(h),
                                      _dp(offset), _dp(old_of_new), _dp(n_out), _stream(stream)),
           "spvar_reduce_noalloc")


ISSUE_FORMS = {0: "lop3", 1: "iadd3", 2: "imad", 3: "mix", 4: "wide", 5: "philox"}


def measure_issue_rate(form, iters, stream=None):
    """Thread-level operations/s of one integer issue probe (see
    spvar_measure_issue_rate) and the timed launch's milliseconds."""
    r, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().spvar_measure_issue_rate(int(form), int(iters), ctypes.byref(r), ctypes.byref(ms),
                                          _stream(stream)), "spvar_measure_issue_rate")
    return r.value, ms.value


def make_params(num_starts=1, fixing_sample_size=100, solving_sample_size=100, num_sweeps=1000, beta0=0.1,
                beta1=3.0, elite_threshold=0.1, fix_num=1, fix_den=1, iterate=False, max_fix_phases=1, canon=-1,
                form=FORM_BATCHED, replicas_per_block=0, sweep_kernel=SWEEP_AUTO, sweep_block=0, start_offset=0,
                component_boost=False, tree_preprocess=False, corr_sample_size=0, corr_elite_threshold=0.2,
                corr_num=1, corr_den=1, sampler=0, sqa_slices=16, sqa_beta=3.0, sqa_gamma0=3.0, sqa_gamma1=0.01,
                sweeps_per_launch=0, pticm_temps=16, pticm_keep=10, pticm_beta0=0.2, pticm_beta1=3.0):
    """Parameters of Alg. 2.  With the PTICM sampler the phase's sample is the
    kept lists, so fixing_sample_size (and a nonzero solving_sample_size) must be
    pticm_sample_size(pticm_temps, pticm_keep)."""
    return Params(num_starts, fixing_sample_size, solving_sample_size, num_sweeps, beta0, beta1, elite_threshold,
                  fix_num, fix_den, 1 if iterate else 0, max_fix_phases, canon, form, replicas_per_block,
                  sweep_kernel, sweep_block, start_offset, 1 if component_boost else 0, 1 if tree_preprocess else 0,
                  corr_sample_size, corr_num, corr_den, float(corr_elite_threshold), sampler, sqa_slices,
                  float(sqa_beta), float(sqa_gamma0), float(sqa_gamma1), int(sweeps_per_launch), int(pticm_temps),
                  int(pticm_keep), float(pticm_beta0), float(pticm_beta1))


def pticm_sample_size(temps, keep):
    """Most states a PTICM phase keeps: K per replica of the lower half of the
    temperatures, two replicas each."""
    return 2 * (temps - temps // 2) * keep


def phase_slots(params):
    """Recorded phase slots: the SPVAR phases, the solving phase and, when
    enabled, the correlation phase."""
    return params.max_fix_phases + 1 + (1 if params.corr_sample_size > 0 else 0)


@dataclasses.dataclass
class SolveOutput:
    energies: object     # [starts, P, Smax]
    counts: object       # [starts, P]
    nfree: object        # [starts, P]
    nphases: object      # [starts]
    fixed: object        # [sum n_p * starts]
    best_energy: object  # [starts]
    best_state: object   # [sum n_p * starts]


def _alloc_outputs(nslots, P, Smax, fm_total, device):
    if device:
        import torch
        mk = lambda shape, dt: torch.empty(shape, dtype=dt, device="cuda")  # noqa: E731
        return SolveOutput(mk((nslots, P, Smax), torch.int64), mk((nslots, P), torch.int32),
                           mk((nslots, P), torch.int32), mk(nslots, torch.int32), mk(max(fm_total, 1), torch.int8),
                           mk(nslots, torch.int64), mk(max(fm_total, 1), torch.int8))
    return SolveOutput(np.zeros((nslots, P, Smax), np.int64), np.zeros((nslots, P), np.int32),
                       np.zeros((nslots, P), np.int32), np.zeros(nslots, np.int32), np.zeros(max(fm_total, 1), np.int8),
                       np.zeros(nslots, np.int64), np.zeros(max(fm_total, 1), np.int8))


def _result_struct(o, device):
    ptr = (lambda t: vp(t.data_ptr())) if device else _hp
    return Result(1 if device else 0, ptr(o.energies), ptr(o.counts), ptr(o.nfree), ptr(o.nphases), ptr(o.fixed),
                  ptr(o.best_energy), ptr(o.best_state))


class Plan:
    """Executable Multi-start SPVAR plan (Alg. 2) over one or more problems."""

    def __init__(self, problems, params, budget_bytes=0, stream=None):
        self.problems = list(problems)
        self.params = params
        arr = (vp * len(self.problems))(*[p.handle for p in self.problems])
        out = vp()
        _check(lib().spvar_plan_create(arr, len(self.problems), ctypes.byref(params), budget_bytes, _stream(stream),
                                       ctypes.byref(out)), "spvar_plan_create")
        self.handle = out
        self.nslots = len(self.problems) * params.num_starts
        self.P = phase_slots(params)
        self.Smax = max(params.fixing_sample_size, params.solving_sample_size, params.corr_sample_size)
        self.fm_total = sum(p.n for p in self.problems) * params.num_starts

    def workspace_bytes(self):
        return int(lib().spvar_plan_workspace_bytes(self.handle))

    def alloc_outputs(self, device=True):
        return _alloc_outputs(self.nslots, self.P, self.Smax, self.fm_total, device)

    def run(self, seeds, out=None, device=True, stream=None):
        seeds = list(seeds) if np.ndim(seeds) else [int(seeds)] * len(self.problems)
        sarr = (u64 * len(seeds))(*[int(s) for s in seeds])
        if out is None:
            out = self.alloc_outputs(device)
        res = _result_struct(out, device)
        _check(lib().spvar_plan_run(self.handle, sarr, ctypes.byref(res), _stream(stream)), "spvar_plan_run")
        return out

    def stats(self):
        a, p = i64(0), i32(0)
        _check(lib().spvar_plan_stats(self.handle, ctypes.byref(a), ctypes.byref(p)), "spvar_plan_stats")
        return a.value, p.value

    def set_profiling(self, on=True):
        _check(lib().spvar_plan_set_profiling(self.handle, 1 if on else 0), "spvar_plan_set_profiling")

    def sweep_time(self):
        ms, n = ctypes.c_double(0), i32(0)
        _check(lib().spvar_plan_sweep_time(self.handle, ctypes.byref(ms), ctypes.byref(n)), "spvar_plan_sweep_time")
        return ms.value, n.value

    def post_time(self):
        """Persistence-pass time (ms) of the last profiled run."""
        ms = ctypes.c_double(0)
        _check(lib().spvar_plan_post_time(self.handle, ctypes.byref(ms)), "spvar_plan_post_time")
        return ms.value

    def shape(self):
        b, r, s, g = i32(0), i32(0), i32(0), i32(0)
        _check(lib().spvar_plan_shape(self.handle, ctypes.byref(b), ctypes.byref(r), ctypes.byref(s), ctypes.byref(g)),
               "spvar_plan_shape")
        spl = i32(0)
        _check(lib().spvar_plan_sweeps_per_launch(self.handle, ctypes.byref(spl)), "spvar_plan_sweeps_per_launch")
        return dict(block=b.value, replicas_per_block=r.value, kernel=("general", "general-staged", "pm1-register", "pm1-streaming", "pm1-warp",
                                                                 "sqa", "sqa-register", "pm1-quads")[s.value],
                    grid=g.value, sweeps_per_launch=spl.value)

    def close(self):
        if self.handle:
            lib().spvar_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(problem, params, seed, device=False, stream=None):
    """One-call Multi-start SPVAR (Alg. 2) of one problem; host outputs by default."""
    nslots = params.num_starts
    P = phase_slots(params)
    Smax = max(params.fixing_sample_size, params.solving_sample_size, params.corr_sample_size)
    out = _alloc_outputs(nslots, P, Smax, problem.n * nslots, device)
    res = _result_struct(out, device)
    _check(lib().spvar_solve(problem.handle, ctypes.byref(params), int(seed), ctypes.byref(res), _stream(stream)),
           "spvar_solve")
    return out


def solve_cache_release():
    """Free the plans that solve() keeps for later calls on problems of the
    same structure with the same parameters."""
    lib().spvar_solve_cache_release()


def unpack_spins(words, n):
    """Bit-packed rows (int32/uint32 [S, W]) -> int8 +-1 [S, n] (host)."""
    w = np.ascontiguousarray(np.asarray(words)).view(np.uint32)
    S = w.shape[0]
    bits = (w[:, :, None] >> np.arange(32, dtype=np.uint32)[None, None, :]) & 1
    return (bits.reshape(S, -1)[:, :n].astype(np.int8) * 2 - 1)


def pack_spins(s):
    """int8 +-1 [S, n] -> uint32 [S, ceil(n/32)] (host)."""
    s = np.asarray(s)
    S, n = s.shape
    W = (n + 31) // 32
    b = np.zeros((S, W * 32), np.uint32)
    b[:, :n] = (s > 0)
    return (b.reshape(S, W, 32) << np.arange(32, dtype=np.uint32)).sum(axis=2).astype(np.uint32)


class Server:
    """Continuous-batching request loop (spvar_server_*): admission by device
    memory budget, one Alg. 2 phase per engine step for everything in flight."""

    def __init__(self, params, budget_bytes, max_n, max_nnz, max_degree, max_dmax, energy_scale=1,
                 max_requests=16, sweeps_per_step=0):
        cfg = ServerConfig(params, int(budget_bytes), max_n, max_nnz, max_degree, max_dmax, energy_scale,
                           max_requests, int(sweeps_per_step))
        out = vp()
        _check(lib().spvar_server_create(ctypes.byref(cfg), ctypes.byref(out)), "spvar_server_create")
        self.handle = out
        self.params = params
        self.P = phase_slots(params)
        self.Smax = max(params.fixing_sample_size, params.solving_sample_size, params.corr_sample_size)
        self.sizes = {}

    def submit(self, inst, seed):
        rp, c, v = csr_from_edges(inst.n, inst.ei, inst.ej, inst.J)
        hh = _host(inst.h, np.int32)
        rid = i64(0)
        _check(lib().spvar_server_submit(self.handle, inst.n, _hp(rp), _hp(c), _hp(v), _hp(hh), int(inst.offset),
                                         int(seed), ctypes.byref(rid)), "spvar_server_submit")
        self.sizes[rid.value] = inst.n
        return rid.value

    def step(self):
        a = i32(0)
        _check(lib().spvar_server_step(self.handle, ctypes.byref(a)), "spvar_server_step")
        return a.value

    def start(self):
        _check(lib().spvar_server_start(self.handle), "spvar_server_start")

    def stop(self):
        _check(lib().spvar_server_stop(self.handle), "spvar_server_stop")

    def info(self, rid, timeout=0.0):
        inf = RequestInfo()
        rc = lib().spvar_server_wait(self.handle, rid, float(timeout), ctypes.byref(inf))
        if rc not in (OK, ETIMEOUT):
            _check(rc, "spvar_server_wait")
        return inf

    def result(self, rid):
        """SolveOutput (host arrays) of a finished request."""
        n, ns = self.sizes[rid], self.params.num_starts
        o = _alloc_outputs(ns, self.P, self.Smax, n * ns, False)
        _check(lib().spvar_server_result(self.handle, rid, _hp(o.best_energy), _hp(o.best_state), _hp(o.fixed),
                                         _hp(o.energies), _hp(o.counts), _hp(o.nfree)), "spvar_server_result")
        return o

    def release(self, rid):
        _check(lib().spvar_server_release(self.handle, rid), "spvar_server_release")

    def stats(self):
        d, a, q, r = i64(0), i64(0), i32(0), i32(0)
        _check(lib().spvar_server_stats(self.handle, ctypes.byref(d), ctypes.byref(a), ctypes.byref(q),
                                        ctypes.byref(r)), "spvar_server_stats")
        return dict(done=d.value, attempts=a.value, queued=q.value, running=r.value)

    def sweep_time(self):
        """(total ms, launches) of the sweep launches of every engine step so far."""
        ms, n = ctypes.c_double(0.0), i64(0)
        _check(lib().spvar_server_sweep_time(self.handle, ctypes.byref(ms), ctypes.byref(n)),
               "spvar_server_sweep_time")
        return ms.value, n.value

    def close(self):
        if self.handle:
            lib().spvar_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
