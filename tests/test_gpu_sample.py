"""GPU parity of the SA sampler (spvar_sample) against the oracle: final
spins and energies must be identical, bit for bit."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I

from gpu_cases import empty, gpu_problem, isolated_spins, oracle_problem, single_spin, table, with_h

pytestmark = pytest.mark.gpu

CASES = [
    ("cubic_L4", lambda: I.cubic3d(4, 1100), 256, 200),
    ("cubic_L5_odd", lambda: I.cubic3d(5, 1101), 37, 150),
    ("chimera_C4", lambda: I.chimera(4, 1200), 50, 150),
    ("weak_strong_C3", lambda: I.weak_strong(3, 1300), 22, 120),
    ("random_general", lambda: I.random_graph(40, 90, 5, jmax=7, hmax=9), 13, 100),
    ("pm1_with_h", lambda: with_h(I.cubic3d(3, 8), 4, 3), 9, 80),
    ("pm1_big_h", lambda: with_h(I.cubic3d(4, 9), 3, 20), 17, 80),
    ("weak_strong_C6", lambda: I.weak_strong(6, 1301), 41, 100),
    ("u10_chimera_C4", lambda: I.chimera_u10(4, 1400), 37, 120),
    ("u10_chimera_C8", lambda: I.chimera_u10(8, 1401), 64, 100),
    ("isolated", isolated_spins, 11, 40),
    ("single_spin", single_spin, 5, 20),
    ("empty", empty, 4, 10),
    ("no_sweeps", lambda: I.cubic3d(3, 2), 6, 0),
]


def _run_both(inst, S, T, seed=12345, start=3, phase=2, r0=0):
    import torch
    from paper_1706_07826_gb300 import spvar
    thr = table(inst, T)
    op = oracle_problem(inst)
    o_spins, o_e, _ = O.sample(op, thr, S, seed, start=start, phase=phase, r0=r0)
    gp = gpu_problem(inst)
    stride = thr.shape[1]
    thr_d = spvar.thresholds_device(thr) if T > 0 else torch.zeros(stride, dtype=torch.int32, device="cuda")
    g_spins, g_e = spvar.sample(gp, thr_d, stride, T, S, seed, start, phase)
    torch.cuda.synchronize()
    return o_spins, o_e + inst.offset, g_spins.cpu().numpy(), g_e.cpu().numpy()


@pytest.mark.parametrize("name,make,S,T", CASES, ids=[c[0] for c in CASES])
def test_sample_parity(cuda_lib, name, make, S, T):
    from paper_1706_07826_gb300 import spvar
    inst = make()
    o_spins, o_e, g_words, g_e = _run_both(inst, S, T)
    assert np.array_equal(g_e[:S], o_e)
    if inst.n:
        assert np.array_equal(spvar.unpack_spins(g_words[:S], inst.n), o_spins)


def test_sample_seed_start_phase_change_the_stream(cuda_lib):
    inst = I.cubic3d(3, 5)
    a = _run_both(inst, 8, 30, seed=1, start=0, phase=0)
    for kw in (dict(seed=2, start=0, phase=0), dict(seed=1, start=1, phase=0), dict(seed=1, start=0, phase=1)):
        b = _run_both(inst, 8, 30, **kw)
        assert np.array_equal(b[1], b[3][:8])  # still bit-exact
        assert not np.array_equal(a[2], b[2])  # and a different stream


def test_chimera_c8_full_size_sampled_replicas(cuda_lib):
    """Chimera C8 (N=512), 1000 samples x 1000 sweeps as the benchmark launches
    them; the oracle recomputes sampled replicas one by one."""
    import torch
    from paper_1706_07826_gb300 import spvar
    inst = I.chimera(8, 1000 + 1 * 100 + 0)
    S, T, seed = 1000, 1000, 42
    thr = table(inst, T)
    gp = gpu_problem(inst)
    g_words, g_e = spvar.sample(gp, spvar.thresholds_device(thr), thr.shape[1], T, S, seed, 0, 0)
    torch.cuda.synchronize()
    g_words, g_e = g_words.cpu().numpy(), g_e.cpu().numpy()
    op = oracle_problem(inst)
    for r in (0, 1, 2, 3, 4, 501, 998, 999):
        s, e, _ = O.sample(op, thr, 1, seed, 0, 0, r0=r)
        assert g_e[r] == e[0], r
        assert np.array_equal(spvar.unpack_spins(g_words[r:r + 1], inst.n)[0], s[0]), r


def test_cubic_L20_unstaged_layout_sampled_replicas(cuda_lib):
    """N = 8000 (the largest served size): the sweep reads its layout from
    global memory instead of shared memory."""
    import torch
    from paper_1706_07826_gb300 import spvar
    inst = I.cubic3d(20, 1500)
    S, T, seed = 64, 100, 7
    thr = table(inst, T)
    gp = gpu_problem(inst)
    g_words, g_e = spvar.sample(gp, spvar.thresholds_device(thr), thr.shape[1], T, S, seed, 1, 0)
    torch.cuda.synchronize()
    op = oracle_problem(inst)
    for r in (0, 33, 63):
        s, e, _ = O.sample(op, thr, 1, seed, 1, 0, r0=r)
        assert g_e[r].item() == e[0]
        assert np.array_equal(spvar.unpack_spins(g_words[r:r + 1].cpu().numpy(), inst.n)[0], s[0])


def test_sample_rejects_short_table(cuda_lib):
    import torch
    from paper_1706_07826_gb300 import spvar
    inst = I.cubic3d(3, 1)
    gp = gpu_problem(inst)
    thr = torch.zeros((5, 4), dtype=torch.int32, device="cuda")  # dmax = 12 needs stride 13
    with pytest.raises(spvar.SpvarError):
        spvar.sample(gp, thr, 4, 5, 8, 1)


@pytest.mark.parametrize("make,S", [(lambda: I.chimera(4, 1200), 37), (lambda: I.cubic3d(20, 1500), 8),
                                    (lambda: I.weak_strong(3, 1300), 13), (lambda: I.cubic3d(5, 1101), 21),
                                    (lambda: I.random_graph(40, 90, 5, jmax=7, hmax=9), 11)],
                         ids=["chimera_register", "cubic_L20_streaming", "weak_strong_register_16bit", "cubic_odd",
                              "random_general"])
def test_resumed_sample_is_identical(cuda_lib, make, S):
    """Checkpoint/resume: sweeps [0, 40) + [40, 97) + [97, 150) from saved states
    equal one uninterrupted 150-sweep sample (and the oracle's)."""
    import torch
    from paper_1706_07826_gb300 import spvar
    inst = make()
    T = 150
    thr = table(inst, T)
    gp = gpu_problem(inst)
    thr_d = spvar.thresholds_device(thr)
    full_s, full_e = spvar.sample(gp, thr_d, thr.shape[1], T, S, 99, 2, 1)
    s1, _ = spvar.sample_range(gp, thr_d, thr.shape[1], 0, 40, S, 99, 2, 1)
    s2, _ = spvar.sample_range(gp, thr_d, thr.shape[1], 40, 97, S, 99, 2, 1, init=s1)
    s3, e3 = spvar.sample_range(gp, thr_d, thr.shape[1], 97, T, S, 99, 2, 1, init=s2)
    torch.cuda.synchronize()
    assert torch.equal(s3, full_s) and torch.equal(e3, full_e)
    if inst.n <= 200:
        o_spins, o_e, _ = O.sample(oracle_problem(inst), thr, S, 99, start=2, phase=1)
        assert np.array_equal(e3.cpu().numpy()[:S], o_e + inst.offset)


def test_resume_edge_cases(cuda_lib):
    """An empty range returns the saved states with their energies; a range
    that does not start at sweep 0 needs saved states, which may not alias the
    output."""
    import torch
    from paper_1706_07826_gb300 import spvar
    inst = I.cubic3d(4, 1102)
    T, S = 60, 20
    thr = table(inst, T)
    gp = gpu_problem(inst)
    thr_d = spvar.thresholds_device(thr)
    s, e = spvar.sample(gp, thr_d, thr.shape[1], T, S, 5)
    s2, e2 = spvar.sample_range(gp, thr_d, thr.shape[1], T, T, S, 5, init=s)
    torch.cuda.synchronize()
    assert torch.equal(s2, s) and torch.equal(e2, e)
    with pytest.raises(spvar.SpvarError):
        spvar.sample_range(gp, thr_d, thr.shape[1], 10, T, S, 5)
    with pytest.raises(spvar.SpvarError):
        spvar.sample_range(gp, thr_d, thr.shape[1], 10, T, S, 5, init=s, spins=s)
    with pytest.raises(spvar.SpvarError):
        spvar.sample_range(gp, thr_d, thr.shape[1], 30, 20, S, 5, init=s)
