"""ctypes wrapper around the C oracle (``spvar_oracle.c``).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Arrays are numpy;
every function mirrors one oracle entry point and cites the step it follows.
"""
import ctypes
import dataclasses

import numpy as np

from . import build as _build

_lib = None

i32p = ctypes.POINTER(ctypes.c_int32)
i64p = ctypes.POINTER(ctypes.c_int64)
u32p = ctypes.POINTER(ctypes.c_uint32)
i8p = ctypes.POINTER(ctypes.c_int8)
f64p = ctypes.POINTER(ctypes.c_double)
u64p = ctypes.POINTER(ctypes.c_uint64)


class OrParams(ctypes.Structure):
    _fields_ = [
        ("num_starts", ctypes.c_int32),
        ("fixing_sample_size", ctypes.c_int32),
        ("solving_sample_size", ctypes.c_int32),
        ("num_sweeps", ctypes.c_int32),
        ("elite_threshold", ctypes.c_double),
        ("fix_num", ctypes.c_int32),
        ("fix_den", ctypes.c_int32),
        ("iterate", ctypes.c_int32),
        ("max_fix_phases", ctypes.c_int32),
        ("canon", ctypes.c_int32),
        ("start0", ctypes.c_int32),
        ("boost", ctypes.c_int32),
        ("tree", ctypes.c_int32),
        ("corr_sample_size", ctypes.c_int32),
        ("corr_num", ctypes.c_int32),
        ("corr_den", ctypes.c_int32),
        ("corr_elite_threshold", ctypes.c_double),
        ("sampler", ctypes.c_int32),
        ("sqa_slices", ctypes.c_int32),
        ("sqa_beta", ctypes.c_double),
        ("sqa_gamma0", ctypes.c_double),
        ("sqa_gamma1", ctypes.c_double),
        ("energy_scale", ctypes.c_int32),
        ("pticm_temps", ctypes.c_int32),
        ("pticm_keep", ctypes.c_int32),
        ("pticm_beta0", ctypes.c_double),
        ("pticm_beta1", ctypes.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_csr_from_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i32p, i32p, i32p]
        L.or_csr_from_edges.restype = ctypes.c_int
        L.or_colour.argtypes = [ctypes.c_int32, i32p, i32p, i32p]
        L.or_colour.restype = ctypes.c_int32
        L.or_dmax.argtypes = [ctypes.c_int32, i32p, i32p, i32p]
        L.or_dmax.restype = ctypes.c_int64
        L.or_thresholds.argtypes = [ctypes.c_int32, f64p, ctypes.c_int32, ctypes.c_int32, u32p]
        L.or_beta_geometric.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, f64p]
        L.or_energy.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i8p]
        L.or_energy.restype = ctypes.c_int64
        L.or_sample.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32,
                                ctypes.c_int32, u32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                ctypes.c_uint32, ctypes.c_uint32, i8p, i64p, i64p]
        L.or_sample.restype = ctypes.c_int
        L.or_sqa_table.argtypes = [ctypes.c_int32, ctypes.c_int32, f64p, f64p, ctypes.c_int32,
                                   ctypes.c_int32, u64p]
        L.or_sqa_sample.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int32, u64p, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, i8p, i64p,
                                    i32p]
        L.or_sqa_sample.restype = ctypes.c_int
        L.or_gamma_linear.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, f64p]
        L.or_icm_move.argtypes = [ctypes.c_int32, i32p, i32p, i8p, i8p, ctypes.c_int32]
        L.or_icm_move.restype = ctypes.c_int32
        L.or_pticm_sample.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, u32p, ctypes.c_int32, u32p, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, i8p, i64p, i32p, i8p, i64p]
        L.or_pticm_sample.restype = ctypes.c_int
        L.or_elite_count.argtypes = [ctypes.c_double, ctypes.c_int32]
        L.or_elite_count.restype = ctypes.c_int32
        L.or_elite.argtypes = [ctypes.c_int32, i64p, ctypes.c_int32, i32p]
        L.or_persistence.argtypes = [ctypes.c_int32, i32p, ctypes.c_int32, i8p, i64p, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, i32p, i8p, i32p]
        L.or_persistence.restype = ctypes.c_int32
        L.or_reduce.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, ctypes.c_int64, i32p, i8p,
                                i32p, i32p, i32p, i32p, i32p, i64p, i32p, i32p]
        L.or_reduce.restype = ctypes.c_int
        L.or_solve.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, ctypes.c_int64,
                               ctypes.POINTER(OrParams), u32p, ctypes.c_int32, ctypes.c_uint64,
                               i64p, i32p, i32p, i32p, i8p, i64p, i8p]
        L.or_solve.restype = ctypes.c_int
        L.or_components.argtypes = [ctypes.c_int32, i32p, i32p, i32p]
        L.or_components.restype = ctypes.c_int32
        L.or_component_boost.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, ctypes.c_int32, i8p, i64p]
        L.or_component_boost.restype = ctypes.c_int
        L.or_tree.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, i64p, i8p, i32p, i32p, i32p]
        L.or_tree.restype = ctypes.c_int32
        L.or_compact.argtypes = [ctypes.c_int32, i32p, i32p, i32p, i32p, ctypes.c_int64, i32p, i8p,
                                 i32p, i32p, i32p, i32p, i32p, i64p, i32p, i32p]
        L.or_compact.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# -- Philox4x32-10 ---------------------------------------------------------
def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: 4 counter words, 2 key words -> 4 words."""
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c, u32p), _p(k, u32p), _p(out, u32p))
    return out


# -- problem ---------------------------------------------------------------
@dataclasses.dataclass
class Csr:
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    h: np.ndarray
    offset: int = 0
    scale: int = 1

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


def csr_from_edges(n, ei, ej, J, h, offset=0, scale=1):
    """Edge list (i != j, each pair once) -> symmetric CSR (Sec. I problem)."""
    ei = _c(ei, np.int32); ej = _c(ej, np.int32); J = _c(J, np.int32)
    m = len(ei)
    rp = np.zeros(n + 1, np.int32)
    col = np.zeros(max(2 * m, 1), np.int32)
    val = np.zeros(max(2 * m, 1), np.int32)
    rc = lib().or_csr_from_edges(n, m, _p(ei, i32p), _p(ej, i32p), _p(J, i32p),
                                 _p(rp, i32p), _p(col, i32p), _p(val, i32p))
    if rc != 0:
        raise ValueError("invalid edge list")
    return Csr(n, rp, col[:2 * m].copy(), val[:2 * m].copy(), _c(h, np.int32).copy(), int(offset), int(scale))


def colour(p: Csr):
    c = np.zeros(max(p.n, 1), np.int32)
    ncol = lib().or_colour(p.n, _p(p.row_ptr, i32p), _p(_c(p.col, np.int32), i32p), _p(c, i32p))
    return c[:p.n].copy(), int(ncol)


def dmax(p: Csr):
    return int(lib().or_dmax(p.n, _p(p.row_ptr, i32p), _p(_c(p.val, np.int32), i32p), _p(p.h, i32p)))


def beta_geometric(T, beta0, beta1):
    b = np.zeros(T, np.float64)
    lib().or_beta_geometric(T, beta0, beta1, _p(b, f64p))
    return b


def thresholds(beta, dmax_, scale=1):
    beta = _c(beta, np.float64)
    T = len(beta)
    thr = np.zeros((T, dmax_ + 1), np.uint32)
    lib().or_thresholds(T, _p(beta, f64p), dmax_, scale, _p(thr, u32p))
    return thr


def energy(p: Csr, s):
    s = _c(s, np.int8)
    return int(lib().or_energy(p.n, _p(p.row_ptr, i32p), _p(_c(p.col, np.int32), i32p),
                               _p(_c(p.val, np.int32), i32p), _p(p.h, i32p), _p(s, i8p)))


def sample(p: Csr, thr, S, seed, start=0, phase=0, colours=None, check_incremental=False, r0=0):
    """SA sample (Sec. III procedure; sampler of the paper's SA runs), replicas r0 .. r0+S-1.

    Returns (spins int8 [S, n] of +-1, energies int64 [S] without offset,
    largest incremental-vs-recomputed energy difference or None)."""
    if colours is None:
        colours = colour(p)
    c, ncol = colours
    thr = _c(thr, np.uint32)
    T = thr.shape[0]
    dm = thr.shape[1] - 1
    spins = np.zeros((max(S, 1), max(p.n, 1)), np.int8)
    e = np.zeros(max(S, 1), np.int64)
    err = np.zeros(1, np.int64)
    c = _c(c, np.int32) if p.n else np.zeros(1, np.int32)
    rc = lib().or_sample(p.n, _p(p.row_ptr, i32p), _p(_c(p.col, np.int32), i32p),
                         _p(_c(p.val, np.int32), i32p), _p(p.h, i32p), _p(c, i32p), ncol,
                         T, _p(thr, u32p), dm, r0, S, seed, start, phase,
                         _p(spins, i8p), _p(e, i64p), _p(err, i64p) if check_incremental else None)
    if rc != 0:
        raise ValueError("or_sample failed: %d" % rc)
    return spins[:S, :p.n].copy(), e[:S].copy(), (int(err[0]) if check_incremental else None)


def sqa_table(T, P, beta, gamma, dmax_, scale=1):
    """SQA acceptance entries [T, 3, 2 (dmax/2) + 1] (uint64; see or_sqa_table).
    beta and gamma: one value per sweep, or a constant."""
    beta = _c(np.broadcast_to(np.asarray(beta, np.float64), (max(T, 1),)), np.float64)
    gamma = _c(np.broadcast_to(np.asarray(gamma, np.float64), (max(T, 1),)), np.float64)
    W = 2 * (dmax_ // 2) + 1
    ent = np.zeros((max(T, 1), 3, W), np.uint64)
    lib().or_sqa_table(T, P, _p(beta, f64p), _p(gamma, f64p), dmax_, scale, _p(ent, u64p))
    return ent[:T]


def gamma_linear(T, gamma0, gamma1):
    """Transverse field falling linearly from gamma0 to gamma1 (endpoints included)."""
    g = np.zeros(max(T, 1), np.float64)
    lib().or_gamma_linear(T, float(gamma0), float(gamma1), _p(g, f64p))
    return g[:T]


def sqa_sample(p: Csr, ent, P, S, seed, start=0, phase=0, colours=None, r0=0):
    """SQA samples (lowest-energy slice of each run): (spins int8 [S, n], e [S], slice [S])."""
    if colours is None:
        colours = colour(p)
    c = _c(colours[0], np.int32) if p.n else np.zeros(1, np.int32)
    ent = _c(ent, np.uint64)
    T = ent.shape[0]
    dmax_ = 2 * ((ent.shape[2] - 1) // 2)
    spins = np.zeros((max(S, 1), max(p.n, 1)), np.int8)
    e = np.zeros(max(S, 1), np.int64)
    sl = np.zeros(max(S, 1), np.int32)
    rc = lib().or_sqa_sample(p.n, _p(p.row_ptr, i32p), _p(_c(p.col, np.int32), i32p), _p(_c(p.val, np.int32), i32p),
                             _p(p.h, i32p), _p(c, i32p), colours[1], T, P, _p(ent, u64p), dmax_, r0, S, seed,
                             start, phase, _p(spins, i8p), _p(e, i64p), _p(sl, i32p))
    if rc != 0:
        raise ValueError("or_sqa_sample failed: %d" % rc)
    return spins[:S, :p.n], e[:S], sl[:S]


def icm_move(p: Csr, a, b, seed_spin):
    """Houdayer's cluster move between replicas a and b (int8 +-1 [n]) seeded at
    seed_spin: returns (a', b', cluster size)."""
    a = _c(a, np.int8).copy()
    b = _c(b, np.int8).copy()
    size = lib().or_icm_move(p.n, _p(p.row_ptr, i32p), _p(_c(p.col, np.int32), i32p), _p(a, i8p), _p(b, i8p),
                             int(seed_spin))
    if size < 0:
        raise ValueError("seed spin outside the set where the replicas differ")
    return a, b, int(size)


def energy_range(p: Csr):
    """An upper bound of max E - min E: 2 (sum_{i<j} |J_ij| + sum_i |h_i|)."""
    return int(np.abs(_c(p.val, np.int64)).sum() + 2 * np.abs(p.h.astype(np.int64)).sum())


def pticm_sample(p: Csr, betas, T, K=10, seed=0, start=0, phase=0, icm_from=None, keep_from=None, exchange=True,
                 icm=True, colours=None):
    """PTICM (Sec. III.D) with the paper's sample: the K lowest-energy distinct
    states seen at each replica of the lower half of the temperatures.  betas:
    R ascending inverse temperatures (problem units).  Returns dict with kept
    [2(R - keep_from), K, n], kept_e, nkept, final [2R, n], final_e (energies
    without offset)."""
    betas = np.asarray(betas, np.float64)
    R = len(betas)
    icm_from = R // 2 if icm_from is None else icm_from
    keep_from = R // 2 if keep_from is None else keep_from
    if colours is None:
        colours = colour(p)
    c = _c(colours[0], np.int32) if p.n else np.zeros(1, np.int32)
    dm = dmax(p)
    thr = np.zeros((R, dm + 1), np.uint32)
    lib().or_thresholds(R, _p(_c(betas, np.float64), f64p), dm, p.scale, _p(thr, u32p))
    dx = max(energy_range(p), 1)
    xthr = np.zeros((max(R - 1, 1), dx + 1), np.uint32)
    if R > 1:
        db = _c(np.diff(betas), np.float64)
        lib().or_thresholds(R - 1, _p(db, f64p), dx, p.scale, _p(xthr, u32p))
    ntr = 2 * (R - keep_from)
    n1 = max(p.n, 1)
    kept = np.zeros((max(ntr, 1), K, n1), np.int8)
    kept_e = np.zeros((max(ntr, 1), K), np.int64)
    nkept = np.zeros(max(ntr, 1), np.int32)
    final = np.zeros((2 * R, n1), np.int8)
    final_e = np.zeros(2 * R, np.int64)
    flags = (1 if exchange else 0) | (2 if icm else 0)
    rc = lib().or_pticm_sample(p.n, _p(p.row_ptr, i32p), _p(_c(p.col, np.int32), i32p),
                               _p(_c(p.val, np.int32), i32p), _p(p.h, i32p), _p(c, i32p), colours[1], R, T,
                               _p(thr, u32p), dm, _p(xthr, u32p), dx, icm_from, keep_from, K, flags, seed, start,
                               phase, _p(kept, i8p), _p(kept_e, i64p), _p(nkept, i32p), _p(final, i8p),
                               _p(final_e, i64p))
    if rc != 0:
        raise ValueError("or_pticm_sample failed: %d" % rc)
    return dict(kept=kept[:ntr, :, :p.n], kept_e=kept_e[:ntr], nkept=nkept[:ntr], final=final[:, :p.n],
                final_e=final_e)


def elite_count(elite, S):
    return int(lib().or_elite_count(float(elite), int(S)))


def elite(e, k):
    e = _c(e, np.int64)
    idx = np.zeros(max(k, 1), np.int32)
    lib().or_elite(len(e), _p(e, i64p), k, _p(idx, i32p))
    return idx[:k].copy()


def persistence(p: Csr, spins, e, k, fix_num=1, fix_den=1, canon=0):
    """Alg. 1 persistence step.  Returns (counts, fixed, nfixed, rho)."""
    spins = _c(spins, np.int8)
    e = _c(e, np.int64)
    S = len(e)
    cnt = np.zeros(max(p.n, 1), np.int32)
    fixed = np.zeros(max(p.n, 1), np.int8)
    rho = np.zeros(1, np.int32)
    nf = lib().or_persistence(p.n, _p(p.row_ptr, i32p), S, _p(spins, i8p), _p(e, i64p), k,
                              fix_num, fix_den, canon, _p(cnt, i32p), _p(fixed, i8p), _p(rho, i32p))
    return cnt[:p.n].copy(), fixed[:p.n].copy(), int(nf), int(rho[0])


def reduce(p: Csr, fixed, colours=None):
    """Alg. 1 update of J and h.  Returns (reduced Csr, colours', old_of_new)."""
    if colours is None:
        colours = colour(p)
    c = _c(colours[0], np.int32) if p.n else np.zeros(1, np.int32)
    fixed = _c(fixed, np.int8) if p.n else np.zeros(1, np.int8)
    n_out = np.zeros(1, np.int32)
    rp = np.zeros(p.n + 1, np.int32)
    col = np.zeros(max(p.nnz, 1), np.int32)
    val = np.zeros(max(p.nnz, 1), np.int32)
    h = np.zeros(max(p.n, 1), np.int32)
    off = np.zeros(1, np.int64)
    co = np.zeros(max(p.n, 1), np.int32)
    oon = np.zeros(max(p.n, 1), np.int32)
    lib().or_reduce(p.n, _p(p.row_ptr, i32p), _p(_c(p.col, np.int32), i32p), _p(_c(p.val, np.int32), i32p),
                    _p(p.h, i32p), p.offset, _p(c, i32p), _p(fixed, i8p), _p(n_out, i32p), _p(rp, i32p),
                    _p(col, i32p), _p(val, i32p), _p(h, i32p), _p(off, i64p), _p(co, i32p), _p(oon, i32p))
    m = int(n_out[0])
    nnz = int(rp[m])
    red = Csr(m, rp[:m + 1].copy(), col[:nnz].copy(), val[:nnz].copy(), h[:m].copy(), int(off[0]), p.scale)
    return red, (co[:m].copy(), colours[1]), oon[:m].copy()


def components(p: Csr):
    """Connected components, numbered by lowest spin index (Sec. II.C)."""
    c = np.zeros(max(p.n, 1), np.int32)
    m = lib().or_components(p.n, _p(p.row_ptr, i32p), _p(_c(p.col, np.int32), i32p), _p(c, i32p))
    return c[:p.n].copy(), int(m)


def component_boost(p: Csr, spins, e):
    """Sec. II.C boosting of a sample; returns (merged spins, merged energies, components)."""
    spins = _c(spins, np.int8).copy()
    e = _c(e, np.int64).copy()
    m = lib().or_component_boost(p.n, _p(p.row_ptr, i32p), _p(_c(p.col, np.int32), i32p),
                                 _p(_c(p.val, np.int32), i32p), _p(p.h, i32p), len(e), _p(spins, i8p), _p(e, i64p))
    return spins, e, int(m)


def tree(p: Csr):
    """Sec. II.C tree pre-processing.  Returns (h', offset', code, parent, order)."""
    h = p.h.copy()
    off = np.array([p.offset], np.int64)
    code = np.zeros(max(p.n, 1), np.int8)
    par = np.zeros(max(p.n, 1), np.int32)
    order = np.zeros(max(p.n, 1), np.int32)
    ninf = np.zeros(1, np.int32)
    lib().or_tree(p.n, _p(p.row_ptr, i32p), _p(_c(p.col, np.int32), i32p), _p(_c(p.val, np.int32), i32p),
                  _p(h, i32p), _p(off, i64p), _p(code, i8p), _p(par, i32p), _p(order, i32p), _p(ninf, i32p))
    return h, int(off[0]), code[:p.n].copy(), par[:p.n].copy(), order[:int(ninf[0])].copy()


def compact(p: Csr, code, colours=None):
    """Drop every spin with code != 0 without folding (after the tree step)."""
    if colours is None:
        colours = colour(p)
    c = _c(colours[0], np.int32) if p.n else np.zeros(1, np.int32)
    code = _c(code, np.int8) if p.n else np.zeros(1, np.int8)
    n_out = np.zeros(1, np.int32)
    rp = np.zeros(p.n + 1, np.int32)
    col = np.zeros(max(p.nnz, 1), np.int32)
    val = np.zeros(max(p.nnz, 1), np.int32)
    h = np.zeros(max(p.n, 1), np.int32)
    off = np.zeros(1, np.int64)
    co = np.zeros(max(p.n, 1), np.int32)
    oon = np.zeros(max(p.n, 1), np.int32)
    lib().or_compact(p.n, _p(p.row_ptr, i32p), _p(_c(p.col, np.int32), i32p), _p(_c(p.val, np.int32), i32p),
                     _p(p.h, i32p), p.offset, _p(c, i32p), _p(code, i8p), _p(n_out, i32p), _p(rp, i32p),
                     _p(col, i32p), _p(val, i32p), _p(h, i32p), _p(off, i64p), _p(co, i32p), _p(oon, i32p))
    m = int(n_out[0])
    nnz = int(rp[m])
    red = Csr(m, rp[:m + 1].copy(), col[:nnz].copy(), val[:nnz].copy(), h[:m].copy(), int(off[0]), p.scale)
    return red, (co[:m].copy(), colours[1]), oon[:m].copy()


@dataclasses.dataclass
class SolveResult:
    energies: np.ndarray   # [starts, P, Smax]
    counts: np.ndarray     # [starts, P]
    nfree: np.ndarray      # [starts, P]
    nphases: np.ndarray    # [starts]
    fixed: np.ndarray      # [starts, n0]
    best_e: np.ndarray     # [starts]
    best_state: np.ndarray # [starts, n0]


def solve(p: Csr, thr, seed, num_starts, fixing_sample_size, solving_sample_size, elite_threshold,
          fix_num=1, fix_den=1, iterate=False, max_fix_phases=1, canon=-1, start0=0, boost=False, tree=False,
          corr_sample_size=0, corr_elite_threshold=0.2, corr_num=1, corr_den=1, sampler=0, sqa_slices=16,
          sqa_beta=3.0, sqa_gamma0=3.0, sqa_gamma1=0.01, pticm_temps=16, pticm_keep=10, pticm_beta0=0.2,
          pticm_beta1=3.0):
    """Multi-start SPVAR (Alg. 2); thr is the original problem's SA table (its
    length sets the sweeps).  corr_sample_size > 0 adds the correlation-fixing
    phase for zero-bias problems; sampler = 1 samples every phase with SQA,
    sampler = 2 with PTICM (the phase's sample is the kept lists; see
    or_params)."""
    thr = _c(thr, np.uint32)
    prm = OrParams(num_starts, fixing_sample_size, solving_sample_size, thr.shape[0], float(elite_threshold),
                   fix_num, fix_den, 1 if iterate else 0, max_fix_phases, canon, start0, 1 if boost else 0,
                   1 if tree else 0, corr_sample_size, corr_num, corr_den, float(corr_elite_threshold), sampler,
                   sqa_slices, float(sqa_beta), float(sqa_gamma0), float(sqa_gamma1), p.scale, pticm_temps,
                   pticm_keep, float(pticm_beta0), float(pticm_beta1))
    P = max_fix_phases + 1 + (1 if corr_sample_size > 0 else 0)
    Smax = max(fixing_sample_size, solving_sample_size, corr_sample_size)
    n0 = p.n
    en = np.zeros((num_starts, P, Smax), np.int64)
    counts = np.zeros((num_starts, P), np.int32)
    nfree = np.zeros((num_starts, P), np.int32)
    nph = np.zeros(num_starts, np.int32)
    fixed = np.zeros((num_starts, max(n0, 1)), np.int8)
    best_e = np.zeros(num_starts, np.int64)
    best_state = np.zeros((num_starts, max(n0, 1)), np.int8)
    rc = lib().or_solve(n0, _p(p.row_ptr, i32p), _p(_c(p.col, np.int32), i32p), _p(_c(p.val, np.int32), i32p),
                        _p(p.h, i32p), p.offset, ctypes.byref(prm), _p(thr, u32p), thr.shape[1] - 1, seed,
                        _p(en, i64p), _p(counts, i32p), _p(nfree, i32p), _p(nph, i32p), _p(fixed, i8p),
                        _p(best_e, i64p), _p(best_state, i8p))
    if rc != 0:
        raise ValueError("or_solve failed: %d" % rc)
    return SolveResult(en, counts, nfree, nph, fixed[:, :n0], best_e, best_state[:, :n0])
