"""Oracle pins for the correlation-fixing step (Sec. II.C: zero-bias problems fix
a cluster of correlated variables instead of one arbitrary variable; Alg. 2
optional step; the appendix gives its own elite threshold, threshold 1.0 and
sample share).

- the step's fixings equal the rule restated here with exact fractions: rho
  (lowest-index spin of maximum degree) fixed to +1, every spin j with
  |mean over the elite of s_rho s_j| >= threshold fixed to the sign;
- it is skipped for a problem with some h != 0 (identical to no step);
- a ferromagnet anneals to its two ground states, so every spin is perfectly
  correlated with rho: all spins end fixed to +1 at the known ground energy;
- fixing rho alone is exact for zero bias (every minimum survives), checked by
  brute force.
"""
import itertools
from fractions import Fraction

import numpy as np

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I


def _csr(inst):
    return O.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J, inst.h, inst.offset, inst.scale)


def _table(p, T):
    return O.thresholds(O.beta_geometric(T, 0.1, 3.0), O.dmax(p), 1)


def _rho(inst):
    deg = np.bincount(np.concatenate([inst.ei, inst.ej]), minlength=inst.n)
    return int(np.flatnonzero(deg == deg.max())[0])


def test_correlation_step_matches_the_rule():
    inst = I.cubic3d(3, 31)
    assert not inst.h.any()
    p = _csr(inst)
    T, Sc, seed = 60, 40, 11
    thr = _table(p, T)
    r = O.solve(p, thr, seed, num_starts=2, fixing_sample_size=30, solving_sample_size=20, elite_threshold=0.2,
                corr_sample_size=Sc, corr_elite_threshold=0.3)
    rho = _rho(inst)
    k = int(np.ceil(0.3 * Sc))
    for st in range(2):
        spins, e, _ = O.sample(p, thr, Sc, seed, start=st, phase=0)
        assert r.counts[st, 0] == Sc
        assert np.array_equal(r.energies[st, 0, :Sc], e + inst.offset)
        elite = np.lexsort((np.arange(Sc), e))[:k]
        corr = {j: Fraction(int((spins[elite, rho] * spins[elite, j]).sum()), k) for j in range(inst.n)}
        fixed = {j: (1 if c > 0 else -1) for j, c in corr.items() if abs(c) >= 1}
        assert fixed[rho] == 1
        assert r.nfree[st, 1] == inst.n - len(fixed)
        for j, v in fixed.items():
            assert r.fixed[st, j] == v
        assert r.nphases[st] == 3 and r.counts[st, 1] == 30 and r.counts[st, 2] == 20


def test_correlation_step_skipped_with_bias():
    inst = I.random_graph(16, 40, 7, jmax=3, hmax=2)
    assert inst.h.any()
    p = _csr(inst)
    thr = _table(p, 50)
    a = O.solve(p, thr, 3, num_starts=2, fixing_sample_size=24, solving_sample_size=12, elite_threshold=0.25)
    b = O.solve(p, thr, 3, num_starts=2, fixing_sample_size=24, solving_sample_size=12, elite_threshold=0.25,
                corr_sample_size=36, corr_elite_threshold=0.3)
    P = a.counts.shape[1]
    assert np.array_equal(a.energies, b.energies[:, :P, :a.energies.shape[2]])
    assert np.array_equal(a.counts, b.counts[:, :P]) and not b.counts[:, P:].any()
    assert np.array_equal(a.fixed, b.fixed) and np.array_equal(a.best_e, b.best_e)


def test_ferromagnet_fixes_every_spin_to_plus():
    base = I.cubic3d(3, 5)
    inst = I.Instance("ferro", base.n, base.ei, base.ej, -np.ones_like(base.J), np.zeros(base.n, np.int32))
    p = _csr(inst)
    thr = _table(p, 200)
    r = O.solve(p, thr, 8, num_starts=2, fixing_sample_size=16, solving_sample_size=8, elite_threshold=0.2,
                corr_sample_size=32, corr_elite_threshold=0.25)
    for st in range(2):
        assert np.all(r.fixed[st] == 1)
        assert r.nfree[st, 1] == 0
        assert r.best_e[st] == -len(inst.J)


def test_fixing_rho_alone_keeps_the_minimum():
    inst = I.random_graph(13, 30, 21, jmax=4, hmax=0)
    assert not inst.h.any()
    p = _csr(inst)
    rho = _rho(inst)
    fx = np.zeros(inst.n, np.int8)
    fx[rho] = 1
    red, _, oon = O.reduce(p, fx)
    S = np.array(list(itertools.product((-1, 1), repeat=inst.n)), np.int64)
    M = np.zeros((inst.n, inst.n), np.int64)
    for a, b, j in zip(inst.ei, inst.ej, inst.J):
        M[min(a, b), max(a, b)] += j
    full_min = np.einsum("si,ij,sj->s", S, M, S).min()
    Sr = S[S[:, rho] == 1][:, oon]
    Mr = np.zeros((red.n, red.n), np.int64)
    for i in range(red.n):
        for q in range(red.row_ptr[i], red.row_ptr[i + 1]):
            if red.col[q] > i:
                Mr[i, red.col[q]] += red.val[q]
    red_min = (np.einsum("si,ij,sj->s", Sr, Mr, Sr) + Sr @ red.h.astype(np.int64)).min() + red.offset
    assert red_min == full_min
