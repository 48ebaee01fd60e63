"""Oracle pins for Alg. 2 with PTICM as the sampler of every phase (Sec.
III.D: the sample of a phase is the K lowest distinct states seen at each
replica of the lower half of the temperatures).

- a phase's recorded sample is the standalone PTICM run's kept lists, list
  after list, with the start's offset, and its size is the number of states
  kept;
- the first phase's fixings are the persistence rule (Alg. 1) applied to that
  sample: elite of ceil(elite * size) states, canonicalised at the reference
  spin for a zero-bias problem, threshold 1, restated here with exact integers;
- every recorded energy is at least the brute-force ground energy, the best
  energy reaches it on small problems, and the best state's dense energy is the
  reported best energy;
- with ISPVAR the phases fix every spin;
- sample sizes that do not match the kept lists are refused.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I


def _csr(inst):
    return O.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J, inst.h, inst.offset, inst.scale)


def _energies(inst, S):
    M = np.zeros((inst.n, inst.n), np.int64)
    for a, b, j in zip(inst.ei, inst.ej, inst.J):
        M[min(a, b), max(a, b)] += j
    S = np.asarray(S, np.int64)
    return np.einsum("ri,ij,rj->r", S, M, S) + S @ inst.h.astype(np.int64) + inst.offset


def _solve(inst, T, R, K, seed, starts=2, **kw):
    p = _csr(inst)
    thr = O.thresholds(O.beta_geometric(T, 0.1, 3.0), O.dmax(p), inst.scale)
    S = 2 * (R - R // 2) * K
    kw.setdefault("solving_sample_size", S)
    return O.solve(p, thr, seed, num_starts=starts, fixing_sample_size=S, elite_threshold=0.25, sampler=2,
                   pticm_temps=R, pticm_keep=K, pticm_beta0=0.3, pticm_beta1=2.5, **kw)


CASES = [("cubic_L3", lambda: I.cubic3d(3, 5)), ("chimera_C2", lambda: I.chimera(2, 6)),
         ("random_h", lambda: I.random_graph(14, 30, 8, jmax=3, hmax=2))]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_phase_sample_is_the_kept_lists_and_fixings_follow_alg1(name, make):
    inst = make()
    inst.offset = 17
    T, R, K, seed = 30, 6, 4, 11
    out = _solve(inst, T, R, K, seed)
    p = _csr(inst)
    betas = np.geomspace(0.3, 2.5, R)
    for st in range(2):
        ref = O.pticm_sample(p, betas, T, K=K, seed=seed, start=st, phase=0)
        kept_e = np.concatenate([ref["kept_e"][q, :ref["nkept"][q]] for q in range(len(ref["nkept"]))])
        kept = np.concatenate([ref["kept"][q, :ref["nkept"][q]] for q in range(len(ref["nkept"]))])
        S = int(ref["nkept"].sum())
        assert out.counts[st, 0] == S
        assert np.array_equal(out.energies[st, 0, :S], kept_e + inst.offset)
        assert np.array_equal(_energies(inst, kept), kept_e + inst.offset)
        # Alg. 1 on that sample: elite by (energy, index), reference-spin canonicalisation
        # when every h is 0, fix where every elite state agrees
        k = max(1, min(S, math.ceil(0.25 * S)))
        order = np.lexsort((np.arange(S), kept_e))[:k]
        E = kept[order].astype(np.int64)
        if not np.any(inst.h):
            deg = np.diff(p.row_ptr)
            rho = int(np.flatnonzero(deg == deg.max())[0])
            E = E * E[:, rho:rho + 1]
        cnt = (E > 0).sum(axis=0)
        want = np.where(cnt == k, 1, np.where(cnt == 0, -1, 0))
        fixed0 = out.fixed[st]
        # phase 0 fixes exactly these (the solving phase fixes nothing)
        assert np.array_equal(fixed0, want)


def test_best_energy_reaches_the_ground_state():
    inst = I.random_graph(12, 26, 21, jmax=3, hmax=3)
    out = _solve(inst, 60, 8, 6, 3, starts=3)
    allS = np.array(list(itertools.product([-1, 1], repeat=inst.n)), np.int64)
    e0 = int(_energies(inst, allS).min())
    for st in range(3):
        c = out.counts[st]
        for ph in range(out.nphases[st]):
            assert np.all(out.energies[st, ph, :c[ph]] >= e0)
        assert out.best_e[st] == e0
        assert _energies(inst, out.best_state[st][None, :])[0] == out.best_e[st]


def test_ispvar_with_pticm_fixes_every_spin():
    inst = I.cubic3d(3, 9)
    out = _solve(inst, 25, 6, 3, 5, starts=2, solving_sample_size=0, iterate=True, max_fix_phases=40)
    for st in range(2):
        assert np.all(out.fixed[st] != 0)
        n = out.nphases[st]
        assert np.all(np.diff(out.nfree[st, :n]) < 0)


def test_sample_sizes_must_match_the_kept_lists():
    inst = I.cubic3d(3, 2)
    p = _csr(inst)
    thr = O.thresholds(O.beta_geometric(10, 0.1, 3.0), O.dmax(p), 1)
    with pytest.raises(ValueError):
        O.solve(p, thr, 1, num_starts=1, fixing_sample_size=10, solving_sample_size=10, elite_threshold=0.2,
                sampler=2, pticm_temps=6, pticm_keep=4)
