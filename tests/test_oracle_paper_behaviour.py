"""Paper-level qualitative pins of the oracle (no GPU): behaviours the paper
reports for its instance classes, reproduced on seeded stand-ins of the same
class.  These pin the method, not numbers the paper prints.

- weak-strong clusters (Sec. III.B): SA ends in the false minimum, where the
  weak cluster is opposite to the strong one, far more often than the
  Boltzmann weight of that state at the final temperature, and a longer
  anneal does not get it out;
- reduced-degeneracy Chimera problems with biases (Sec. III.C, couplers and
  biases from U_10): one SPVAR phase fixes most of the variables.  The paper
  reports more than 80 % with its quantum annealer as the sampler; SA at 1000
  sweeps and 100 samples fixes a median of about 73 % on C8 (48 % to 83 % over
  ten seeds), so the pin is a median above 60 % over five problems.
"""
import itertools

import numpy as np

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I


def _csr(inst):
    return O.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J, inst.h, inst.offset, inst.scale)


def test_weak_strong_pair_false_minimum():
    inst = I.weak_strong_pair()
    p = _csr(inst)
    S = np.array(list(itertools.product((-1, 1), repeat=inst.n)), np.int64)
    M = np.zeros((inst.n, inst.n), np.int64)
    for a, b, j in zip(inst.ei, inst.ej, inst.J):
        M[a, b] += j
    E = np.einsum("si,ij,sj->s", S, M, S) + S @ inst.h.astype(np.int64)
    strong_up = np.all(S[:, :8] == 1, axis=1)
    e_gs = E.min()
    e_false = E[strong_up & np.all(S[:, 8:] == -1, axis=1)][0]
    assert E[strong_up & np.all(S[:, 8:] == 1, axis=1)][0] == e_gs  # ground state: both clusters aligned
    assert e_false > e_gs
    # Boltzmann weight of the false minimum against the ground state at the final beta
    beta1 = 3.0
    w_false = np.exp(-beta1 * (e_false - e_gs) / inst.scale)
    for T in (1000, 4000):
        thr = O.thresholds(O.beta_geometric(T, 0.1, beta1), O.dmax(p), inst.scale)
        s, e, _ = O.sample(p, thr, 400, 7)
        in_false = np.mean(e == e_false)
        assert np.all((e == e_gs) | (e == e_false) | (e > e_false))
        assert in_false > 0.25 and in_false > 4 * w_false, (T, in_false, w_false)


def test_spvar_fixes_most_variables_on_u10_chimera():
    T = 1000
    fixed = []
    for seed in range(2500, 2505):
        inst = I.chimera_u10(8, seed)
        p = _csr(inst)
        thr = O.thresholds(O.beta_geometric(T, 0.1, 3.0), O.dmax(p), inst.scale)
        r = O.solve(p, thr, 5, num_starts=1, fixing_sample_size=100, solving_sample_size=10, elite_threshold=0.1)
        fixed.append(1 - r.nfree[0, 1] / inst.n)  # phase 1 is the solving phase on the reduced problem
    assert np.median(fixed) > 0.6, fixed
