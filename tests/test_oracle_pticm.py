"""Oracle pins for PTICM, parallel tempering with isoenergetic cluster moves
(Sec. III.D), with the paper's sample rule (the lowest-energy distinct states
seen at each replica of the lower half of the temperatures).

- without exchanges and cluster moves every replica is the SA oracle at its
  constant temperature, bit for bit (same random words and decisions);
- the cluster move is Houdayer's: the flipped set equals the connected
  component of the seed among the spins where the two replicas differ
  (scipy), both replicas flip on it, the pair's total energy is unchanged,
  and each copy's energy moves by -+2 times the cluster's boundary sum;
- the whole chain (Metropolis, cluster moves, exchanges) leaves each
  temperature's Boltzmann distribution in place: chi-square of the final
  states of many independent runs against enumeration, at both temperatures;
- the kept lists hold distinct states with their true energies, in order, and
  at the coldest replica of a small problem they are the lowest energies of
  the whole state space (brute force);
- a run reaches the brute-force ground state.
"""
import itertools

import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components
from scipy.stats import chi2 as chi2d

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


def test_metropolis_part_is_simulated_annealing():
    inst = I.random_graph(14, 30, 3, jmax=3, hmax=2)
    p = _csr(inst)
    betas = np.array([0.3, 0.9, 2.0])
    T, seed, start, phase = 25, 91, 4, 2
    r = O.pticm_sample(p, betas, T, K=3, seed=seed, start=start, phase=phase, exchange=False, icm=False)
    for k, b in enumerate(betas):
        thr = O.thresholds(np.full(T, b), O.dmax(p), inst.scale)
        for c in range(2):
            s, e, _ = O.sample(p, thr, 1, seed, start=start, phase=phase, r0=2 * k + c)
            assert np.array_equal(r["final"][2 * k + c], s[0]) and r["final_e"][2 * k + c] == e[0]


def test_cluster_move_is_houdayers():
    inst = I.random_graph(24, 40, 5, jmax=4, hmax=3)
    p = _csr(inst)
    A = csr_matrix((np.ones(len(inst.ei)), (inst.ei, inst.ej)), shape=(inst.n, inst.n))
    A = A + A.T
    g = np.random.default_rng(7)
    for _ in range(60):
        a = g.choice([-1, 1], inst.n).astype(np.int8)
        b = g.choice([-1, 1], inst.n).astype(np.int8)
        D = np.flatnonzero(a != b)
        if len(D) == 0:
            continue
        seed_spin = int(g.choice(D))
        a2, b2, size = O.icm_move(p, a, b, seed_spin)
        _, lab = connected_components(A[D][:, D], directed=False)
        cluster = D[lab == lab[np.searchsorted(D, seed_spin)]]
        flipped = np.flatnonzero(a2 != a)
        assert np.array_equal(flipped, cluster) and size == len(cluster)
        assert np.array_equal(np.flatnonzero(b2 != b), cluster)
        assert np.array_equal(a2[cluster], b[cluster]) and np.array_equal(b2[cluster], a[cluster])
        assert _E(inst, a2)[0] + _E(inst, b2)[0] == _E(inst, a)[0] + _E(inst, b)[0]
        # each copy's change is -+2 (sum over the cluster of h_i a_i and of J_ij a_i a_j over the couplers
        # leaving it): every such coupler ends outside D, where the copies agree
        inC = np.zeros(inst.n, bool)
        inC[cluster] = True
        ai = a.astype(np.int64)
        bnd = int((inst.h[cluster] * ai[cluster]).sum())
        for i, j, w in zip(inst.ei, inst.ej, inst.J):
            if inC[i] != inC[j]:
                assert a[i] == b[i] and not inC[i] or a[j] == b[j] and not inC[j]
                bnd += int(w) * int(ai[i]) * int(ai[j])
        assert _E(inst, a2)[0] - _E(inst, a)[0] == -2 * bnd
        assert _E(inst, b2)[0] - _E(inst, b)[0] == 2 * bnd
    with pytest.raises(ValueError):
        same = np.ones(inst.n, np.int8)
        O.icm_move(p, same, same, 0)


def test_chain_keeps_boltzmann_at_every_temperature():
    inst = I.random_graph(5, 7, 11, jmax=2, hmax=2)
    p = _csr(inst)
    betas = np.array([0.4, 1.1])
    runs, T = 12000, 30
    cols = O.colour(p)
    states = {0: [], 1: []}
    for run in range(runs):
        r = O.pticm_sample(p, betas, T, K=1, seed=5, start=run, icm_from=1, keep_from=1, colours=cols)
        for k in (0, 1):
            states[k].append(r["final"][2 * k])
    S = np.array(list(itertools.product((-1, 1), repeat=inst.n)), np.int64)
    E = _E(inst, S)
    code_of = {tuple(s): i for i, s in enumerate(S)}
    for k, b in enumerate(betas):
        w = np.exp(-b * (E - E.min()))
        w /= w.sum()
        obs = np.bincount([code_of[tuple(np.asarray(s, np.int64))] for s in states[k]], minlength=len(S))
        exp = w * runs
        keep = exp >= 5
        stat = (((obs[keep] - exp[keep]) ** 2) / exp[keep]).sum()
        assert obs[~keep].sum() <= max(20.0, 3 * exp[~keep].sum())
        assert chi2d.sf(stat, keep.sum() - 1) > 1e-3, (k, stat)


def test_kept_states_are_the_lowest_seen():
    inst = I.random_graph(8, 14, 13, jmax=3, hmax=2)
    p = _csr(inst)
    betas = np.geomspace(0.3, 1.5, 4)
    K = 10
    r = O.pticm_sample(p, betas, 3000, K=K, seed=17)
    S = np.array(list(itertools.product((-1, 1), repeat=inst.n)), np.int64)
    lowest = np.sort(_E(inst, S))[:K]
    assert len(r["nkept"]) == 2 * (len(betas) - len(betas) // 2)
    for q in range(len(r["nkept"])):
        nk = r["nkept"][q]
        kept, ke = r["kept"][q, :nk], r["kept_e"][q, :nk]
        assert np.array_equal(_E(inst, kept), ke)
        assert np.all(np.diff(ke) >= 0)
        assert len({tuple(s) for s in kept}) == nk
    coldest = len(r["nkept"]) - 2
    assert r["nkept"][coldest] == K and np.array_equal(r["kept_e"][coldest], lowest)


def test_reaches_ground_state():
    inst = I.random_graph(16, 34, 23, jmax=3, hmax=2)
    p = _csr(inst)
    S = np.array(list(itertools.product((-1, 1), repeat=inst.n)), np.int64)
    e0 = _E(inst, S).min()
    r = O.pticm_sample(p, np.geomspace(0.2, 3.0, 8), 400, K=10, seed=29)
    assert r["kept_e"][:, 0].min() == e0
