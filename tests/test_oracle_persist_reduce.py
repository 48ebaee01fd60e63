"""Oracle pins for the persistence pass and fold/compact (Alg. 1) and for the
Multi-start loop (Alg. 2).

- elite order against numpy's lexsort; k = ceil(elite * S);
- counts and the fixing rule against exact rational arithmetic;
- the zero-bias canonicalisation is invariant under flipping any elite row;
- reduction invariant: E_full(s) = E_reduced(s_free) + offset' for every
  assignment consistent with the fixings (exhaustive for n <= 14);
- solve: recorded energies are valid energies (>= brute-force minimum) and the
  best state's energy, recomputed densely, equals the reported best energy.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I


def _csr(inst):
    return O.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J, inst.h, inst.offset, inst.scale)


def _dense(inst):
    M = np.zeros((inst.n, inst.n), np.int64)
    for a, b, j in zip(inst.ei, inst.ej, inst.J):
        M[min(a, b), max(a, b)] += j
    return M


def _E(inst, S):
    S = np.atleast_2d(np.asarray(S, np.int64))
    return np.einsum("si,ij,sj->s", S, _dense(inst), S) + S @ inst.h.astype(np.int64) + inst.offset


def _E_csr(p, S):
    """Energy of a Csr problem (incl. offset) through a dense matrix built here."""
    S = np.atleast_2d(np.asarray(S, np.int64))
    M = np.zeros((p.n, p.n), np.int64)
    for i in range(p.n):
        for q in range(p.row_ptr[i], p.row_ptr[i + 1]):
            if p.col[q] > i:
                M[i, p.col[q]] += p.val[q]
    return np.einsum("si,ij,sj->s", S, M, S) + S @ p.h.astype(np.int64) + p.offset


@pytest.mark.parametrize("S,elite,k", [(256, 0.1, 26), (1000, 0.1, 100), (250, 0.2, 50), (7, 1.0, 7),
                                       (5, 1e-9, 1), (2000, 0.1, 200), (500, 0.3, 150)])
def test_elite_count(S, elite, k):
    assert O.elite_count(elite, S) == k


def test_elite_order_matches_lexsort():
    g = np.random.default_rng(1)
    e = g.integers(-20, 5, 300).astype(np.int64)  # many ties
    for k in (1, 17, 300):
        ref = np.lexsort((np.arange(300), e))[:k]
        assert np.array_equal(O.elite(e, k), ref)


@pytest.mark.parametrize("canon", [0, 1])
@pytest.mark.parametrize("tau", [(1, 1), (9, 10), (1, 2)])
def test_persistence_counts_and_rule(canon, tau):
    inst = I.random_graph(20, 45, 4)
    p = _csr(inst)
    g = np.random.default_rng(2)
    S = 60
    spins = np.where(g.random((S, 20)) < 0.8, 1, -1).astype(np.int8)
    spins[:, 3] = 1
    spins[:, 5] = -1
    e = g.integers(-10, 10, S).astype(np.int64)
    k = 13
    cnt, fixed, nf, rho = O.persistence(p, spins, e, k, tau[0], tau[1], canon)
    idx = np.lexsort((np.arange(S), e))[:k]
    rows = spins[idx].astype(np.int64)
    deg = np.diff(p.row_ptr)
    if canon:
        assert rho == int(np.argmax(deg))
        rows = rows * rows[:, rho:rho + 1]
    else:
        assert rho == -1
    assert np.array_equal(cnt, (rows > 0).sum(axis=0))
    for i in range(20):
        mean = Fraction(int(rows[:, i].sum()), k)
        want = int(np.sign(mean.numerator)) if abs(mean) >= Fraction(tau[0], tau[1]) else 0
        assert fixed[i] == want
    assert nf == int((fixed != 0).sum())


def test_canonicalisation_breaks_zero_bias_degeneracy():
    inst = I.cubic3d(3, 2)
    p = _csr(inst)
    g = np.random.default_rng(5)
    base = np.where(g.random(inst.n) < 0.5, 1, -1).astype(np.int8)
    S = 40
    spins = np.array([base if r % 2 == 0 else -base for r in range(S)], np.int8)
    e = np.zeros(S, np.int64)
    _, fixed0, nf0, _ = O.persistence(p, spins, e, S, 1, 1, 0)
    assert nf0 == 0                      # each state appears with its reverse: nothing persists
    _, fixed1, nf1, rho = O.persistence(p, spins, e, S, 1, 1, 1)
    assert nf1 == inst.n                 # up to the global flip every row is the same state
    assert np.array_equal(fixed1, base * base[rho])
    flipped = spins.copy()
    flipped[[1, 6, 7]] *= -1             # flipping elite rows changes nothing under canon
    assert np.array_equal(O.persistence(p, flipped, e, S, 1, 1, 1)[1], fixed1)


def _all_consistent(n, fixed):
    free = np.flatnonzero(fixed == 0)
    out = np.tile(fixed.astype(np.int64), (2 ** len(free), 1))
    if len(free):
        out[:, free] = np.array(list(itertools.product([-1, 1], repeat=len(free))), np.int64)
    return out, free


@pytest.mark.parametrize("pattern", ["none", "all", "one", "random", "half"])
def test_reduction_invariant_exhaustive(pattern):
    inst = I.random_graph(13, 30, 9, jmax=4, hmax=3)
    inst.offset = 17
    p = _csr(inst)
    g = np.random.default_rng(11)
    fixed = {"none": np.zeros(13), "all": g.choice([-1, 1], 13), "one": np.eye(13)[4] * -1,
             "random": g.choice([-1, 0, 1], 13), "half": np.where(np.arange(13) % 2, 1, 0)}[pattern].astype(np.int8)
    red, (col2, _), oon = O.reduce(p, fixed)
    S, free = _all_consistent(13, fixed)
    assert np.array_equal(oon, free)
    assert red.n == len(free)
    full = _E(inst, S)
    sub = _E_csr(red, S[:, free]) if red.n else np.full(len(S), red.offset)
    assert np.array_equal(full, sub)
    colours, _ = O.colour(p)
    assert np.array_equal(col2, colours[free])


def test_reduction_invariant_sampled_scaled_problem():
    inst = I.weak_strong(3, 6)
    p = _csr(inst)
    g = np.random.default_rng(12)
    fixed = g.choice([-1, 0, 0, 1], inst.n).astype(np.int8)
    red, _, oon = O.reduce(p, fixed)
    S = g.choice([-1, 1], (10000, inst.n)).astype(np.int64)
    S[:, fixed != 0] = fixed[fixed != 0]
    assert np.array_equal(_E(inst, S), _E_csr(red, S[:, oon]))
    # the reduced CSR stays symmetric with ascending columns
    for i in range(red.n):
        cols = red.col[red.row_ptr[i]:red.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0)


def test_solve_energies_are_valid_and_best_state_consistent():
    inst = I.random_graph(14, 36, 13, jmax=3, hmax=1)
    p = _csr(inst)
    thr = O.thresholds(O.beta_geometric(150, 0.1, 3.0), O.dmax(p), 1)
    r = O.solve(p, thr, seed=5, num_starts=4, fixing_sample_size=24, solving_sample_size=16,
                elite_threshold=0.25)
    allS, _ = _all_consistent(14, np.zeros(14, np.int8))
    e0 = _E(inst, allS).min()
    for st in range(4):
        assert r.nphases[st] == 2
        assert list(r.counts[st]) == [24, 16]
        assert r.nfree[st, 0] == 14 and r.nfree[st, 1] <= 14
        rec = np.concatenate([r.energies[st, ph, :r.counts[st, ph]] for ph in range(2)])
        assert rec.min() >= e0
        assert r.best_e[st] == rec.min()
        assert _E(inst, r.best_state[st])[0] == r.best_e[st]
        assert 14 - r.nfree[st, 1] == int((r.fixed[st] != 0).sum())


def test_ispvar_fixes_every_spin():
    inst = I.cubic3d(3, 21)
    p = _csr(inst)
    thr = O.thresholds(O.beta_geometric(100, 0.1, 3.0), O.dmax(p), 1)
    r = O.solve(p, thr, seed=9, num_starts=2, fixing_sample_size=32, solving_sample_size=0,
                elite_threshold=0.1, iterate=True, max_fix_phases=inst.n)
    for st in range(2):
        assert np.all(r.fixed[st] != 0)
        ph = r.nphases[st]
        assert np.all(np.diff(r.nfree[st, :ph]) < 0)   # every phase fixes at least one spin
        assert _E(inst, r.best_state[st])[0] == r.best_e[st]


def _disconnected():
    """Three pieces: a 3D L=3 lattice, a Chimera cell, and two isolated biased spins."""
    a, b = I.cubic3d(3, 14), I.chimera(1, 15)
    n = a.n + b.n + 2
    ei = np.concatenate([a.ei, b.ei + a.n])
    ej = np.concatenate([a.ej, b.ej + a.n])
    J = np.concatenate([a.J, b.J])
    h = np.zeros(n, np.int32)
    h[-2:] = [3, -2]
    h[:5] = [1, 0, -1, 2, 0]
    return I.Instance("disconnected", n, ei.astype(np.int32), ej.astype(np.int32), J.astype(np.int32), h)


def test_components_against_scipy():
    import scipy.sparse as sp
    from scipy.sparse import csgraph
    inst = _disconnected()
    p = _csr(inst)
    comp, m = O.components(p)
    A = sp.csr_matrix((np.ones(p.nnz), p.col, p.row_ptr), shape=(p.n, p.n))
    m2, lab = csgraph.connected_components(A, directed=False)
    assert m == m2 == 4
    # same partition, numbered by lowest member
    first = {}
    for i, l in enumerate(lab):
        first.setdefault(l, len(first))
    assert np.array_equal(comp, np.array([first[l] for l in lab]))


def test_component_boost_invariants():
    inst = _disconnected()
    p = _csr(inst)
    thr = O.thresholds(O.beta_geometric(20, 0.1, 1.0), O.dmax(p), 1)
    spins, e, _ = O.sample(p, thr, 40, seed=3)
    ms, me, m = O.component_boost(p, spins, e)
    assert m == 4
    # every merged state is a valid assignment whose energy is the merged energy
    assert np.array_equal(_E(inst, ms), me)
    # ranks: non-decreasing energies; the best merged state is at least as good as the best state
    assert np.all(np.diff(me) >= 0)
    assert me[0] <= e.min()
    comp, _ = O.components(p)
    # rank 0 takes each component's best partial state: its energy is the sum of the minima
    M = _dense(inst)
    S64 = spins.astype(np.int64)
    best_sum = 0
    for c in range(4):
        sel = comp == c
        Mc = M[np.ix_(sel, sel)]
        part = np.einsum("si,ij,sj->s", S64[:, sel], Mc, S64[:, sel]) + S64[:, sel] @ inst.h[sel].astype(np.int64)
        best_sum += part.min()
    assert me[0] == best_sum


def test_component_boost_is_a_sort_on_connected_problems():
    inst = I.chimera(2, 8)
    p = _csr(inst)
    thr = O.thresholds(O.beta_geometric(10, 0.1, 1.0), O.dmax(p), 1)
    spins, e, _ = O.sample(p, thr, 30, seed=4)
    ms, me, m = O.component_boost(p, spins, e)
    assert m == 1
    order = np.lexsort((np.arange(30), e))
    assert np.array_equal(me, e[order])
    assert np.array_equal(ms, spins[order])


def test_solve_with_boost_only_improves_the_solving_phase():
    inst = I.cubic3d(4, 31)
    p = _csr(inst)
    thr = O.thresholds(O.beta_geometric(40, 0.1, 3.0), O.dmax(p), 1)
    kw = dict(num_starts=3, fixing_sample_size=64, solving_sample_size=40, elite_threshold=0.1, fix_num=3,
              fix_den=4)
    a = O.solve(p, thr, seed=2, **kw)
    b = O.solve(p, thr, seed=2, boost=True, **kw)
    for st in range(3):
        assert np.array_equal(a.energies[st, 0], b.energies[st, 0])          # fixing phase untouched
        sa, sb = a.energies[st, 1, :40], b.energies[st, 1, :40]
        assert np.all(np.diff(sb) >= 0) and sb[0] <= sa.min()
        assert b.best_e[st] <= a.best_e[st]
        assert _E(inst, b.best_state[st])[0] == b.best_e[st]


def _tree_reconstruct(full_n, free_idx, s_free, code, parent, order, J_of):
    """Full assignment from a reduced one: fixed codes, free values, inferred last-first."""
    s = np.zeros(full_n, np.int64)
    s[code == 1], s[code == -1] = 1, -1
    s[free_idx] = s_free
    for i in order[::-1]:
        s[i] = -np.sign(J_of(i, parent[i])) * s[parent[i]]
    return s


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_tree_preprocessing_is_exact(seed):
    """Every reduced assignment lifts to a full one with E_full = E_reduced + offset',
    and the minimum is preserved (brute force), on sparse problems with trees."""
    g = np.random.default_rng(seed)
    n = 12
    inst = I.random_graph(n, 13 + seed, 100 + seed, jmax=4, hmax=3)
    if seed == 4:
        inst.h[:] = 0  # zero bias: only inference and arbitrary degree-0 fixings
    p = _csr(inst)
    h2, off2, code, parent, order = O.tree(p)
    assert len(order) == int((code == 2).sum())
    p2 = O.Csr(p.n, p.row_ptr, p.col, p.val, h2, off2, p.scale)
    red, _, oon = O.compact(p2, code)
    assert red.n == int((code == 0).sum())
    J = {(int(a), int(b)): int(v) for a, b, v in zip(inst.ei, inst.ej, inst.J)}
    J_of = lambda i, j: J.get((i, j), J.get((j, i)))
    allS = np.array(list(itertools.product([-1, 1], repeat=n)), np.int64)
    e_min = _E(inst, allS).min()
    if red.n:
        sub = np.array(list(itertools.product([-1, 1], repeat=red.n)), np.int64)
        e_red = _E_csr(red, sub)
    else:
        sub = np.zeros((1, 0), np.int64)
        e_red = np.array([red.offset])
    for k in range(len(sub)):
        s = _tree_reconstruct(n, oon, sub[k], code, parent, order, J_of)
        assert _E(inst, s)[0] == e_red[k]
    assert e_red.min() == e_min


def test_tree_eliminates_whole_trees():
    # a path 0-1-2-3 and a star centred at 4 with leaves 5,6,7: everything goes
    ei = np.array([0, 1, 2, 4, 4, 4], np.int32)
    ej = np.array([1, 2, 3, 5, 6, 7], np.int32)
    inst = I.Instance("forest", 8, ei, ej, np.array([2, -3, 1, 1, -1, 2], np.int32), np.array([1, 0, 0, -1, 0, 0, 0, 0], np.int32))
    h2, off2, code, parent, order = O.tree(_csr(inst))
    assert np.all(code != 0)
    allS = np.array(list(itertools.product([-1, 1], repeat=8)), np.int64)
    assert off2 == _E(inst, allS).min()


def test_solve_with_tree_states_are_consistent():
    inst = I.random_graph(40, 48, 17, jmax=3, hmax=2)
    p = _csr(inst)
    thr = O.thresholds(O.beta_geometric(60, 0.1, 3.0), O.dmax(p), 1)
    r = O.solve(p, thr, seed=4, num_starts=3, fixing_sample_size=32, solving_sample_size=24,
                elite_threshold=0.2, tree=True)
    r0 = O.solve(p, thr, seed=4, num_starts=3, fixing_sample_size=32, solving_sample_size=24,
                 elite_threshold=0.2)
    for st in range(3):
        assert _E(inst, r.best_state[st])[0] == r.best_e[st]
        assert np.array_equal(r.energies[st, 0], r0.energies[st, 0])   # the first sample is untouched
        assert r.nfree[st, 1] <= r0.nfree[st, 1]                        # trees only shrink the problem
