"""Shared helpers of the GPU parity tests: problem construction on both sides
from one seeded instance (no value ever flows from the CUDA path to the
oracle)."""
import numpy as np

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I


def oracle_problem(inst):
    return O.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J, inst.h, inst.offset, inst.scale)


def gpu_problem(inst):
    from paper_1706_07826_gb300 import spvar
    return spvar.Problem.from_instance(inst)


def table(inst, T, beta0=0.1, beta1=3.0, dmax=None):
    p = oracle_problem(inst)
    d = O.dmax(p) if dmax is None else dmax
    return O.thresholds(O.beta_geometric(T, beta0, beta1), d, inst.scale) if T > 0 else np.zeros((0, d + 1), np.uint32)


def with_h(inst, seed, hmax):
    g = np.random.default_rng(seed)
    inst.h = g.integers(-hmax, hmax + 1, inst.n).astype(np.int32)
    return inst


def single_spin():
    return I.Instance("single", 1, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32),
                      np.array([3], np.int32))


def empty():
    return I.Instance("empty", 0, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32),
                      np.zeros(0, np.int32), offset=5)


def isolated_spins():
    inst = I.random_graph(12, 6, 77, jmax=2, hmax=2)  # several isolated vertices
    return inst
