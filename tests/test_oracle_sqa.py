"""Oracle pins for the second sampler: simulated quantum annealing (discrete-time
path-integral Monte Carlo of the transverse-field Ising model, Sec. III).

- one Trotter slice is classical: SQA with P = 1 and the SA schedule is the
  SA oracle, bit for bit (same random words, same order, same decisions);
- the acceptance entries against the flip cost of the path-integral action
  recomputed here from its definition by brute force (sum over slices of the
  classical energies and of the slice couplings), for random configurations;
- at a constant field and temperature the output distribution (lowest-energy
  slice of each run, and which slice) follows exp(-A) summed over all 2^(nP)
  path configurations (chi-square);
- a slow anneal reaches the brute-force ground state of a small problem;
- recorded energies are the energies of the returned states.
"""
import itertools

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
    return np.einsum("si,ij,sj->s", S, _dense(inst), S) + S @ inst.h.astype(np.int64)


def _action(inst, X, beta, gamma, P):
    """A(x) for path configurations X [..., P, n] (without the offset)."""
    X = np.asarray(X, np.int64)
    E = np.stack([_E(inst, X[:, tau]) for tau in range(P)], axis=1) / inst.scale
    A = beta / P * E.sum(axis=1)
    if P > 1:
        jp = -0.5 * np.log(np.tanh(beta * gamma / P))
        A -= jp * (X * np.roll(X, -1, axis=1)).sum(axis=(1, 2))
    return A


@pytest.mark.parametrize("make", [lambda: I.cubic3d(3, 5), lambda: I.chimera(2, 6),
                                  lambda: I.random_graph(20, 50, 7, jmax=4, hmax=3), lambda: I.weak_strong(1, 8)],
                         ids=["cubic", "chimera", "random_h", "weak_strong_scaled"])
def test_single_slice_is_simulated_annealing(make):
    inst = make()
    p = _csr(inst)
    T = 40
    beta = O.beta_geometric(T, 0.1, 3.0)
    thr = O.thresholds(beta, O.dmax(p), inst.scale)
    ent = O.sqa_table(T, 1, beta, 0.7, O.dmax(p), inst.scale)
    s1, e1, _ = O.sample(p, thr, 9, 77, start=3, phase=1)
    s2, e2, sl = O.sqa_sample(p, ent, 1, 9, 77, start=3, phase=1)
    assert np.array_equal(s1, s2) and np.array_equal(e1, e2) and not sl.any()


def test_entries_follow_the_action():
    inst = I.random_graph(5, 8, 3, jmax=2, hmax=2)
    p = _csr(inst)
    dmax = O.dmax(p)
    bias = dmax // 2
    P, beta, gamma = 4, 0.9, np.array([2.5, 0.4])
    ent = O.sqa_table(2, P, beta, gamma, dmax, 1)
    g = np.random.default_rng(1)
    for _ in range(200):
        t = int(g.integers(2))
        X = g.choice([-1, 1], size=(1, P, inst.n))
        tau, i = int(g.integers(P)), int(g.integers(inst.n))
        Y = X.copy()
        Y[0, tau, i] *= -1
        dA = (_action(inst, Y, beta, gamma[t], P) - _action(inst, X, beta, gamma[t], P))[0]
        dE = int(_E(inst, Y[:, tau])[0] - _E(inst, X[:, tau])[0])
        a = int(X[0, (tau + 1) % P, i] == X[0, tau, i]) + int(X[0, (tau - 1) % P, i] == X[0, tau, i])
        thr = (1 << 32) - int(ent[t, a, dE // 2 + bias])
        want = min(1.0, np.exp(-dA)) * 2.0 ** 32
        assert abs(thr - want) <= 1e-6 * 2.0 ** 32 + 1
        assert (ent[t, a, dE // 2 + bias] == 0) == (dA <= 1e-12)
    # more aligned slice neighbours and larger classical cost never make a flip likelier
    assert np.all(np.diff(ent.astype(np.float64), axis=1) >= 0)
    assert np.all(np.diff(ent.astype(np.float64), axis=2) >= 0)


def test_output_distribution_at_constant_field():
    inst = I.Instance("tri", 3, np.array([0, 0, 1], np.int32), np.array([1, 2, 2], np.int32),
                      np.array([1, 1, -1], np.int32), np.array([1, 0, -1], np.int32))
    p = _csr(inst)
    P, beta, gamma, T, S = 4, 0.7, 2.0, 300, 8000
    ent = O.sqa_table(T, P, beta, gamma, O.dmax(p), 1)
    spins, e, sl = O.sqa_sample(p, ent, P, S, seed=2024)
    # exact: enumerate every path configuration, weight exp(-A), map to (state, slice)
    X = np.array(list(itertools.product((-1, 1), repeat=P * inst.n)), np.int64).reshape(-1, P, inst.n)
    w = np.exp(-_action(inst, X, beta, gamma, P))
    w /= w.sum()
    E = np.stack([_E(inst, X[:, tau]) for tau in range(P)], axis=1)
    best = np.argmin(E, axis=1)  # first minimum = lowest slice on ties
    state_code = ((X[np.arange(len(X)), best] > 0) * (1 << np.arange(inst.n))).sum(axis=1)
    bins = state_code * P + best
    expected = np.bincount(bins, weights=w, minlength=8 * P) * S
    got_code = ((spins > 0) * (1 << np.arange(inst.n))).sum(axis=1)
    observed = np.bincount(got_code * P + sl, minlength=8 * P).astype(np.float64)
    keep = expected >= 5
    assert observed[~keep].sum() <= max(20.0, 3 * expected[~keep].sum())
    chi2 = (((observed[keep] - expected[keep]) ** 2) / expected[keep]).sum()
    from scipy.stats import chi2 as chi2d
    assert chi2d.sf(chi2, keep.sum() - 1) > 1e-3, chi2


def test_slow_anneal_reaches_ground_state():
    inst = I.random_graph(12, 26, 5, jmax=3, hmax=2)
    p = _csr(inst)
    allS = np.array(list(itertools.product((-1, 1), repeat=inst.n)), np.int64)
    e0 = _E(inst, allS).min()
    T, P = 400, 8
    ent = O.sqa_table(T, P, 4.0, O.gamma_linear(T, 3.0, 0.05), O.dmax(p), 1)
    spins, e, sl = O.sqa_sample(p, ent, P, 16, seed=9)
    assert e.min() == e0
    assert np.array_equal(_E(inst, spins), e)
    assert np.all((sl >= 0) & (sl < P))


def test_odd_slice_count_rejected():
    inst = I.cubic3d(3, 1)
    p = _csr(inst)
    ent = O.sqa_table(3, 3, 1.0, 1.0, O.dmax(p), 1)
    with pytest.raises(ValueError):
        O.sqa_sample(p, ent, 3, 4, 1)


def test_solve_with_one_slice_equals_constant_temperature_sa():
    """Alg. 2 with the SQA sampler at P = 1 and inverse temperature beta is
    Alg. 2 with SA at the constant schedule beta0 = beta1 = beta."""
    inst = I.random_graph(18, 40, 11, jmax=3, hmax=2)
    p = _csr(inst)
    T, beta = 60, 1.7
    thr = O.thresholds(O.beta_geometric(T, beta, beta), O.dmax(p), 1)
    kw = dict(num_starts=3, fixing_sample_size=20, solving_sample_size=12, elite_threshold=0.25)
    a = O.solve(p, thr, 5, **kw)
    b = O.solve(p, thr, 5, sampler=1, sqa_slices=1, sqa_beta=beta, sqa_gamma0=1.0, sqa_gamma1=0.5, **kw)
    for f in ("energies", "counts", "nfree", "nphases", "fixed", "best_e", "best_state"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_solve_with_sqa_records_valid_energies():
    inst = I.random_graph(14, 30, 13, jmax=3, hmax=1)
    p = _csr(inst)
    T = 80
    thr = O.thresholds(O.beta_geometric(T, 0.1, 3.0), O.dmax(p), 1)
    r = O.solve(p, thr, 6, num_starts=2, fixing_sample_size=16, solving_sample_size=8, elite_threshold=0.25,
                sampler=1, sqa_slices=4, sqa_beta=3.0, sqa_gamma0=2.0, sqa_gamma1=0.05)
    allS = np.array(list(itertools.product((-1, 1), repeat=inst.n)), np.int64)
    e0 = _E(inst, allS).min()
    for st in range(2):
        rec = np.concatenate([r.energies[st, ph, :r.counts[st, ph]] for ph in range(r.nphases[st])])
        assert rec.min() >= e0 and r.best_e[st] == rec.min()
        assert _E(inst, r.best_state[st])[0] == r.best_e[st]
