"""Oracle pins for the simulated-annealing sampler (Sec. III.A).

- the running energy equals a full recomputation after every sweep;
- at beta = 0 every proposal is accepted, so s_T = (-1)^T s_0;
- at a fixed beta the sampled states follow the Boltzmann distribution
  (chi-square against brute-force enumeration);
- long anneals reach the brute-force ground energy on small problems;
- a ferromagnet anneals to one of its two uniform ground states;
- the acceptance table matches its definition evaluated with numpy.
"""
import itertools

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I


def _csr(inst):
    return O.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J, inst.h, inst.offset, inst.scale)


def _all_states(n):
    return np.array(list(itertools.product([-1, 1], repeat=n)), np.int64)


def _energies_dense(inst, S):
    M = np.zeros((inst.n, inst.n), np.int64)
    for a, b, j in zip(inst.ei, inst.ej, inst.J):
        M[min(a, b), max(a, b)] += j
    return np.einsum("si,ij,sj->s", S, M, S) + S @ inst.h.astype(np.int64)


def _table(p, beta):
    return O.thresholds(beta, O.dmax(p), p.scale)


@pytest.mark.parametrize("inst", [I.random_graph(14, 40, 11, jmax=5, hmax=4), I.weak_strong(2, 3),
                                  I.cubic3d(3, 4), I.chimera(2, 5)], ids=lambda x: x.name)
def test_incremental_energy_equals_recomputed(inst):
    p = _csr(inst)
    thr = _table(p, O.beta_geometric(60, 0.1, 3.0))
    spins, e, err = O.sample(p, thr, 9, seed=77, check_incremental=True)
    assert err == 0
    for r in range(9):
        assert O.energy(p, spins[r]) == e[r]


def test_beta_zero_flips_every_spin_every_sweep():
    inst = I.random_graph(10, 20, 2)
    p = _csr(inst)
    s0, _, _ = O.sample(p, _table(p, np.zeros(0)), 13, seed=5)
    for T in (1, 2, 3, 8):
        sT, _, _ = O.sample(p, _table(p, np.zeros(T)), 13, seed=5)
        assert np.array_equal(sT, s0 * (-1) ** T)


def test_threshold_table_definition():
    beta = np.array([0.0, 0.1, 0.7, 3.0, 50.0])
    thr = O.thresholds(beta, 12, 1)
    ref = np.minimum(np.floor(np.ldexp(np.exp(-beta[:, None] * np.arange(13)[None, :]), 32)), 2.0 ** 32 - 1)
    assert np.array_equal(thr.astype(np.float64), ref)
    thr100 = O.thresholds(beta, 300, 100)
    ref100 = np.minimum(np.floor(np.ldexp(np.exp(-beta[:, None] * np.arange(301)[None, :] / 100.0), 32)),
                        2.0 ** 32 - 1)
    assert np.array_equal(thr100.astype(np.float64), ref100)


def test_beta_schedule_endpoints():
    b = O.beta_geometric(1000, 0.1, 3.0)
    assert b[0] == 0.1 and abs(b[-1] - 3.0) < 1e-12
    assert np.allclose(np.diff(np.log(b)), np.log(30.0) / 999)


@pytest.mark.parametrize("inst,beta", [(I.random_graph(6, 9, 21, jmax=2, hmax=2), 0.6),
                                       (I.weak_strong(1, 8), 0.3)], ids=["random6", "weakstrong8"])
def test_fixed_beta_samples_are_boltzmann(inst, beta):
    p = _csr(inst)
    T = 40
    S = 120000
    spins, _, _ = O.sample(p, _table(p, np.full(T, beta)), S, seed=2024)
    states = _all_states(inst.n)
    E = _energies_dense(inst, states)
    w = np.exp(-beta * (E - E.min()) / inst.scale)
    prob = w / w.sum()
    code = ((spins > 0).astype(np.int64) * (1 << np.arange(inst.n - 1, -1, -1))).sum(axis=1)
    obs = np.bincount(code, minlength=len(states))
    # itertools.product order is big-endian in +1 bits
    keep = prob * S > 5
    exp = prob * S
    chi = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum() + 0.0
    pval = stats.chi2.sf(chi, keep.sum() - 1)
    assert pval > 1e-3, (chi, keep.sum())
    assert obs[~keep].sum() <= max(10, 3 * exp[~keep].sum())


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_long_anneal_reaches_brute_force_ground_state(seed):
    inst = I.random_graph(16, 40, seed, jmax=3, hmax=2)
    p = _csr(inst)
    E = _energies_dense(inst, _all_states(inst.n))
    spins, e, _ = O.sample(p, _table(p, O.beta_geometric(1500, 0.1, 5.0)), 32, seed=seed)
    assert e.min() == E.min()
    assert e.min() >= E.min()


def test_ferromagnet_reaches_uniform_ground_state():
    inst = I.cubic3d(3, 9)
    inst.J[:] = -1
    p = _csr(inst)
    spins, e, _ = O.sample(p, _table(p, O.beta_geometric(800, 0.1, 3.0)), 8, seed=3)
    best = int(np.argmin(e))
    assert e[best] == -3 * inst.n
    assert abs(int(spins[best].sum())) == inst.n
