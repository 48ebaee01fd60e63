"""GPU parity of the persistence pass (spvar_persistence) and of fold/compact
(spvar_reduce) against the oracle: elite order, counts, fixings, reduced CSR,
fields, offset, colours and sweep order must match exactly."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I

from gpu_cases import gpu_problem, oracle_problem, table, with_h

pytestmark = pytest.mark.gpu

PCASES = [
    ("cubic_L4_h0_canon", lambda: I.cubic3d(4, 1100), 256, 80, 0.1, (1, 1), -1),
    ("chimera_C4_h0_nocanon", lambda: I.chimera(4, 1200), 101, 80, 0.2, (1, 1), 0),
    ("weak_strong_tau09", lambda: I.weak_strong(3, 1300), 64, 80, 0.3, (9, 10), -1),
    ("random_k_all", lambda: I.random_graph(30, 60, 9, jmax=4, hmax=3), 17, 60, 1.0, (1, 1), -1),
    ("pm1_h_canon_forced", lambda: with_h(I.cubic3d(3, 8), 4, 2), 40, 60, 0.25, (3, 4), 1),
]


def _samples(inst, S, T, seed):
    import torch
    from paper_1706_07826_gb300 import spvar
    thr = table(inst, T)
    op = oracle_problem(inst)
    o_spins, o_e, _ = O.sample(op, thr, S, seed)
    gp = gpu_problem(inst)
    g_words, g_e = spvar.sample(gp, spvar.thresholds_device(thr), thr.shape[1], T, S, seed)
    torch.cuda.synchronize()
    return op, o_spins, o_e + inst.offset, gp, g_words, g_e


@pytest.mark.parametrize("name,make,S,T,elite,tau,canon", PCASES, ids=[c[0] for c in PCASES])
def test_persistence_parity(cuda_lib, name, make, S, T, elite, tau, canon):
    from paper_1706_07826_gb300 import spvar
    inst = make()
    op, o_spins, o_e, gp, g_words, g_e = _samples(inst, S, T, seed=99)
    k = O.elite_count(elite, S)
    c = canon if canon >= 0 else int(not np.any(inst.h))
    o_cnt, o_fix, o_nf, _ = O.persistence(op, o_spins, o_e, k, tau[0], tau[1], c)
    g_elite, g_cnt, g_fix, g_nf, g_k = spvar.persistence(gp, S, g_words, g_e, elite, tau[0], tau[1], canon)
    assert g_k == k
    assert np.array_equal(g_elite.cpu().numpy(), O.elite(o_e, k))
    assert np.array_equal(g_cnt.cpu().numpy(), o_cnt)
    assert np.array_equal(g_fix.cpu().numpy(), o_fix)
    assert int(g_nf.item()) == o_nf


def _compare_problem(gp, red, colours):
    d = gp.download()
    assert d["n"] == red.n
    assert np.array_equal(d["row_ptr"], red.row_ptr)
    assert np.array_equal(d["col"], red.col)
    assert np.array_equal(d["val"], red.val)
    assert np.array_equal(d["h"], red.h)
    assert d["offset"] == red.offset
    assert np.array_equal(d["colour"], colours[0])


RCASES = [
    ("cubic_L5_random", lambda: I.cubic3d(5, 3), "random"),
    ("weak_strong_C3_random", lambda: I.weak_strong(3, 4), "random"),
    ("chimera_C3_none", lambda: I.chimera(3, 5), "none"),
    ("chimera_C3_all", lambda: I.chimera(3, 6), "all"),
    ("random_dense_h", lambda: I.random_graph(50, 200, 7, jmax=9, hmax=9), "random"),
]


@pytest.mark.parametrize("name,make,pattern", RCASES, ids=[c[0] for c in RCASES])
def test_reduce_parity_then_sample_reduced(cuda_lib, name, make, pattern):
    import torch
    from paper_1706_07826_gb300 import spvar
    inst = make()
    inst.offset = -11
    op = oracle_problem(inst)
    g = np.random.default_rng(21)
    fixed = {"random": g.choice([-1, 0, 0, 1], inst.n), "none": np.zeros(inst.n),
             "all": g.choice([-1, 1], inst.n)}[pattern].astype(np.int8)
    red, colours, oon = O.reduce(op, fixed)
    gp = gpu_problem(inst)
    g_red, g_oon = spvar.reduce(gp, torch.from_numpy(fixed).cuda())
    assert np.array_equal(g_oon.cpu().numpy(), oon)
    _compare_problem(g_red, red, colours)
    # the reduced problem's sweep layout drives an identical anneal
    T, S = 60, 21
    thr = table(inst, T)  # the original table covers every reduction
    o_spins, o_e, _ = O.sample(red, thr, S, 5, colours=colours)
    g_words, g_e = spvar.sample(g_red, spvar.thresholds_device(thr), thr.shape[1], T, S, 5)
    torch.cuda.synchronize()
    assert np.array_equal(g_e.cpu().numpy()[:S], o_e + red.offset)
    if red.n:
        assert np.array_equal(spvar.unpack_spins(g_words.cpu().numpy()[:S], red.n), o_spins)
    # and a second level of reduction
    fixed2 = g.choice([-1, 0, 1], red.n).astype(np.int8)
    red2, colours2, oon2 = O.reduce(red, fixed2, colours)
    g_red2, g_oon2 = spvar.reduce(g_red, torch.from_numpy(fixed2).cuda() if red.n else
                                  torch.zeros(1, dtype=torch.int8, device="cuda"))
    assert np.array_equal(g_oon2.cpu().numpy(), oon2)
    _compare_problem(g_red2, red2, colours2)
