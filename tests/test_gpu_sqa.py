"""GPU parity of the second sampler, simulated quantum annealing
(spvar_sqa_sample, discrete-time path integral, Sec. III), against the
oracle: returned states, energies and chosen slices identical, bit for bit,
for +-1 and general couplers, one to sixteen Trotter slices, and sampled
replicas of a full-size Chimera C8 run."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I

from gpu_cases import gpu_problem, oracle_problem, table, with_h

pytestmark = pytest.mark.gpu

CASES = [
    # name, instance, P, T, S
    ("cubic_L4_P4", lambda: I.cubic3d(4, 2100), 4, 60, 37),
    ("cubic_L5_odd_P8", lambda: I.cubic3d(5, 2101), 8, 40, 22),
    ("chimera_C3_P2", lambda: I.chimera(3, 2102), 2, 50, 16),
    ("chimera_C2_P16", lambda: I.chimera(2, 2103), 16, 30, 9),
    ("pm1_with_h_P6", lambda: with_h(I.cubic3d(3, 2104), 4, 3), 6, 40, 13),
    ("random_general_P4", lambda: I.random_graph(40, 90, 5, jmax=7, hmax=9), 4, 40, 11),
    ("weak_strong_scaled_P8", lambda: I.weak_strong(2, 2105), 8, 30, 8),
    ("u10_C3_P4", lambda: I.chimera_u10(3, 2130), 4, 40, 16),
    ("u10_C4_P8", lambda: I.chimera_u10(4, 2131), 8, 30, 12),
    ("single_slice", lambda: I.cubic3d(4, 2106), 1, 50, 20),
]


def _gpu(inst, P, ent, S, seed, start, phase):
    import torch
    from paper_1706_07826_gb300 import spvar
    g, e, sl = spvar.sqa_sample(gpu_problem(inst), spvar.table_device(ent), ent.shape[2], ent.shape[0], P, S, seed,
                                start, phase)
    torch.cuda.synchronize()
    return spvar.unpack_spins(g.cpu().numpy()[:S], inst.n), e.cpu().numpy()[:S], sl.cpu().numpy()[:S]


@pytest.mark.parametrize("name,make,P,T,S", CASES, ids=[c[0] for c in CASES])
def test_sqa_parity(cuda_lib, name, make, P, T, S):
    inst = make()
    op = oracle_problem(inst)
    ent = O.sqa_table(T, P, 3.0, O.gamma_linear(T, 3.0, 0.05), O.dmax(op), inst.scale)
    o_s, o_e, o_sl = O.sqa_sample(op, ent, P, S, 321, start=2, phase=1)
    g_s, g_e, g_sl = _gpu(inst, P, ent, S, 321, 2, 1)
    assert np.array_equal(g_e, o_e + inst.offset)
    assert np.array_equal(g_sl, o_sl)
    assert np.array_equal(g_s, o_s)


def test_single_slice_equals_sa_kernel(cuda_lib):
    import torch
    from paper_1706_07826_gb300 import spvar
    inst = I.chimera(4, 2107)
    op = oracle_problem(inst)
    T, S = 80, 24
    beta = O.beta_geometric(T, 0.1, 3.0)
    thr = table(inst, T)
    ent = O.sqa_table(T, 1, beta, 1.0, O.dmax(op), 1)
    gp = gpu_problem(inst)
    w1, e1 = spvar.sample(gp, spvar.thresholds_device(thr), thr.shape[1], T, S, 5, 1, 0)
    torch.cuda.synchronize()
    s2, e2, sl = _gpu(inst, 1, ent, S, 5, 1, 0)
    assert np.array_equal(e1.cpu().numpy()[:S], e2) and not sl.any()
    assert np.array_equal(spvar.unpack_spins(w1.cpu().numpy()[:S], inst.n), s2)


def test_chimera_c8_sampled_replicas(cuda_lib):
    """Chimera C8 (N = 512) with 16 slices, 64 runs; the oracle recomputes
    sampled runs one by one."""
    inst = I.chimera(8, 2108)
    op = oracle_problem(inst)
    T, P, S = 60, 16, 64
    ent = O.sqa_table(T, P, 3.0, O.gamma_linear(T, 3.0, 0.05), O.dmax(op), 1)
    g_s, g_e, g_sl = _gpu(inst, P, ent, S, 99, 0, 0)
    for r in (0, 5, 31, 63):
        s, e, sl = O.sqa_sample(op, ent, P, 1, 99, r0=r)
        assert g_e[r] == e[0] and g_sl[r] == sl[0]
        assert np.array_equal(g_s[r], s[0])


def test_sqa_rejects_bad_arguments(cuda_lib):
    from paper_1706_07826_gb300 import spvar
    inst = I.cubic3d(4, 1)
    op = oracle_problem(inst)
    ent = O.sqa_table(10, 4, 1.0, 1.0, O.dmax(op), 1)
    gp = gpu_problem(inst)
    d = spvar.table_device(ent)
    with pytest.raises(spvar.SpvarError):
        spvar.sqa_sample(gp, d, ent.shape[2], 10, 3, 8, 1)            # odd slice count
    with pytest.raises(spvar.SpvarError):
        spvar.sqa_sample(gp, d, ent.shape[2] - 2, 10, 4, 8, 1)        # table narrower than the problem's dmax
    big = I.cubic3d(20, 2)
    gb = gpu_problem(big)
    eb = O.sqa_table(2, 1024, 1.0, 1.0, O.dmax(oracle_problem(big)), 1)
    with pytest.raises(spvar.SpvarError):
        spvar.sqa_sample(gb, spvar.table_device(eb), eb.shape[2], 2, 1024, 4, 1)  # slices do not fit


SOLVE = [
    # name, instance, P, T, starts, S_fix, S_solve, elite, extra
    ("chimera_C3_P4", lambda: I.chimera(3, 2110), 4, 40, 3, 40, 24, 0.2, {}),
    ("cubic_L4_P8_ispvar", lambda: I.cubic3d(4, 2111), 8, 30, 2, 32, 0, 0.1, dict(iterate=True, max_fix_phases=6)),
    ("random_h_P2_tree_boost", lambda: I.random_graph(40, 60, 7, jmax=3, hmax=2), 2, 40, 2, 32, 20, 0.25,
     dict(tree=True, boost=True)),
    ("weak_strong_P8_corr_skip", lambda: I.weak_strong(2, 2112), 8, 30, 2, 24, 16, 0.2, dict(corr_sample_size=16)),
    ("cubic_L4_P4_corr", lambda: I.cubic3d(4, 2113), 4, 30, 2, 24, 16, 0.2, dict(corr_sample_size=20)),
]


@pytest.mark.parametrize("form", [0, 1], ids=["batched", "plain"])
@pytest.mark.parametrize("name,make,P,T,starts,Sf,Ss,elite,extra", SOLVE, ids=[c[0] for c in SOLVE])
def test_solve_with_sqa_parity(cuda_lib, form, name, make, P, T, starts, Sf, Ss, elite, extra):
    """Alg. 2 with the SQA sampler in every phase: identical to the oracle."""
    from paper_1706_07826_gb300 import spvar
    inst = make()
    op = oracle_problem(inst)
    okw = dict(extra)
    gkw = {{"tree": "tree_preprocess", "boost": "component_boost"}.get(k, k): v for k, v in extra.items()}
    sq = dict(sqa_slices=P, sqa_beta=3.0, sqa_gamma0=2.5, sqa_gamma1=0.05)
    ref = O.solve(op, table(inst, T), 31, num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss,
                  elite_threshold=elite, sampler=1, **sq, **okw)
    prm = spvar.make_params(num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss, num_sweeps=T,
                            elite_threshold=elite, form=form, sampler=spvar.SAMPLER_SQA, **sq, **gkw)
    out = spvar.solve(gpu_problem(inst), prm, 31)
    for s in range(starts):
        assert int(out.nphases[s]) == ref.nphases[s]
        assert np.array_equal(np.asarray(out.counts[s]), ref.counts[s])
        assert np.array_equal(np.asarray(out.nfree[s]), ref.nfree[s])
        for ph in range(ref.nphases[s]):
            c = ref.counts[s, ph]
            assert np.array_equal(np.asarray(out.energies[s, ph, :c]), ref.energies[s, ph, :c]), (s, ph)
        assert int(out.best_energy[s]) == ref.best_e[s]
        n = inst.n
        assert np.array_equal(np.asarray(out.fixed[s * n:(s + 1) * n]), ref.fixed[s])
        assert np.array_equal(np.asarray(out.best_state[s * n:(s + 1) * n]), ref.best_state[s])


def test_sqa_sampler_parameters_validated(cuda_lib):
    from paper_1706_07826_gb300 import spvar
    gp = gpu_problem(I.chimera(2, 3))
    for kw in (dict(sampler=2), dict(sampler=1, sqa_slices=3), dict(sampler=1, sqa_gamma1=0.0),
               dict(sampler=1, sqa_beta=-1.0)):
        with pytest.raises(spvar.SpvarError):
            spvar.solve(gp, spvar.make_params(num_starts=1, fixing_sample_size=8, solving_sample_size=8,
                                              num_sweeps=10, **kw), 1)


REQUESTED = [
    # kernel, block, expected shape name
    ("PM1S", 128, "sqa"),
    ("PM1S", 512, "sqa"),
    ("PM1", 256, "sqa-register"),
    ("PM1", 512, "sqa-register"),
    ("PM1", 1024, "sqa-register"),
    ("GENERAL", 256, "sqa"),
]
REQ_CASES = [
    ("chimera_C3_P4", lambda: I.chimera(3, 2120), 4, 30, 3, 24, 16, 0.2, {}),
    ("cubic_L5_odd_3col_P8_h", lambda: with_h(I.cubic3d(5, 2121), 3, 5), 8, 20, 2, 16, 8, 0.25, {}),
    ("cubic_L4_P2_ispvar", lambda: I.cubic3d(4, 2122), 2, 20, 2, 16, 0, 0.2, dict(iterate=True, max_fix_phases=4)),
]


@pytest.mark.parametrize("kernel,block,shape", REQUESTED, ids=["%s_%d" % r[:2] for r in REQUESTED])
@pytest.mark.parametrize("name,make,P,T,starts,Sf,Ss,elite,extra", REQ_CASES, ids=[c[0] for c in REQ_CASES])
def test_solve_with_sqa_requested_kernel(cuda_lib, kernel, block, shape, name, make, P, T, starts, Sf, Ss, elite,
                                         extra):
    """Every SQA sweep variant (item walk, register form at 256/512/1024
    threads, general path), requested explicitly: Alg. 2 identical to the
    oracle in every phase."""
    from paper_1706_07826_gb300 import spvar
    inst = make()
    op = oracle_problem(inst)
    sq = dict(sqa_slices=P, sqa_beta=3.0, sqa_gamma0=2.5, sqa_gamma1=0.05)
    ref = O.solve(op, table(inst, T), 41, num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss,
                  elite_threshold=elite, sampler=1, **sq, **extra)
    prm = spvar.make_params(num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss, num_sweeps=T,
                            elite_threshold=elite, sampler=spvar.SAMPLER_SQA, replicas_per_block=4,
                            sweep_kernel=getattr(spvar, "SWEEP_" + kernel), sweep_block=block, **sq, **extra)
    plan = spvar.Plan([gpu_problem(inst)], prm)
    assert plan.shape()["kernel"] == shape and plan.shape()["block"] == block
    out = plan.run([41], device=False)
    plan.close()
    for s in range(starts):
        assert int(out.nphases[s]) == ref.nphases[s]
        assert np.array_equal(np.asarray(out.counts[s]), ref.counts[s])
        for ph in range(ref.nphases[s]):
            c = ref.counts[s, ph]
            assert np.array_equal(np.asarray(out.energies[s, ph, :c]), ref.energies[s, ph, :c]), (s, ph)
        n = inst.n
        assert int(out.best_energy[s]) == ref.best_e[s]
        assert np.array_equal(np.asarray(out.fixed[s * n:(s + 1) * n]), ref.fixed[s])
        assert np.array_equal(np.asarray(out.best_state[s * n:(s + 1) * n]), ref.best_state[s])


def test_sqa_register_form_rejections(cuda_lib):
    """The register form needs every colour class to fit the block; the warp
    kernel has no SQA form."""
    from paper_1706_07826_gb300 import spvar
    gp = gpu_problem(I.cubic3d(10, 2123))  # two classes of 500 spins
    base = dict(num_starts=1, fixing_sample_size=8, solving_sample_size=8, num_sweeps=10, sampler=spvar.SAMPLER_SQA,
                sqa_slices=4, sqa_beta=3.0, sqa_gamma0=2.0, sqa_gamma1=0.1, replicas_per_block=4)
    # 256 threads: falls back to the item walk
    plan = spvar.Plan([gp], spvar.make_params(sweep_kernel=spvar.SWEEP_PM1, sweep_block=256, **base))
    assert plan.shape()["kernel"] == "sqa"
    plan.close()
    plan = spvar.Plan([gp], spvar.make_params(sweep_kernel=spvar.SWEEP_PM1, sweep_block=512, **base))
    assert plan.shape()["kernel"] == "sqa-register"
    plan.close()
    with pytest.raises(spvar.SpvarError):
        spvar.Plan([gp], spvar.make_params(sweep_kernel=spvar.SWEEP_PM1W, sweep_block=256, **base))


def test_cubic_L12_sampled_replicas_block_1024(cuda_lib):
    """3D L = 12 (N = 1728, two colour classes of 864 spins: the register form
    at 1024 threads), 4 slices, 40 runs; sampled runs recomputed by the oracle."""
    inst = I.cubic3d(12, 2124)
    op = oracle_problem(inst)
    T, P, S = 30, 4, 40
    ent = O.sqa_table(T, P, 3.0, O.gamma_linear(T, 3.0, 0.05), O.dmax(op), 1)
    g_s, g_e, g_sl = _gpu(inst, P, ent, S, 77, 1, 2)
    for r in (0, 13, 39):
        s, e, sl = O.sqa_sample(op, ent, P, 1, 77, start=1, phase=2, r0=r)
        assert g_e[r] == e[0] + inst.offset and g_sl[r] == sl[0]
        assert np.array_equal(g_s[r], s[0])


def test_sqa_register_form_with_never_accept_entries(cuda_lib):
    """A transverse field that ends near zero makes the slice coupling so
    strong that some moves are never accepted (entry 2^32): the register form
    then keeps 64-bit entries, and Alg. 2 stays identical to the oracle."""
    from paper_1706_07826_gb300 import spvar
    inst = I.chimera(3, 2125)
    op = oracle_problem(inst)
    T, P = 30, 8
    sq = dict(sqa_slices=P, sqa_beta=3.0, sqa_gamma0=2.0, sqa_gamma1=1e-7)
    ent = O.sqa_table(T, P, 3.0, O.gamma_linear(T, 2.0, 1e-7), O.dmax(op), 1)
    assert (ent == 1 << 32).any()
    kw = dict(num_starts=2, fixing_sample_size=24, solving_sample_size=16, elite_threshold=0.2)
    ref = O.solve(op, table(inst, T), 43, sampler=1, **sq, **kw)
    prm = spvar.make_params(num_sweeps=T, sampler=spvar.SAMPLER_SQA, replicas_per_block=4,
                            sweep_kernel=spvar.SWEEP_PM1, sweep_block=256, **sq, **kw)
    plan = spvar.Plan([gpu_problem(inst)], prm)
    assert plan.shape()["kernel"] == "sqa-register"
    out = plan.run([43], device=False)
    plan.close()
    for s in range(2):
        for ph in range(ref.nphases[s]):
            c = ref.counts[s, ph]
            assert np.array_equal(np.asarray(out.energies[s, ph, :c]), ref.energies[s, ph, :c]), (s, ph)
        assert np.array_equal(np.asarray(out.best_state[s * inst.n:(s + 1) * inst.n]), ref.best_state[s])


def test_sqa_autotune_cache_keeps_each_tables_entry_width(cuda_lib):
    """Two autotuned plans of the same geometry share the tuned shape, but the
    second one's table has never-accept entries: it must not inherit 32-bit
    entries from the first."""
    from paper_1706_07826_gb300 import spvar
    inst = I.chimera(3, 2126)
    op = oracle_problem(inst)
    T, P = 30, 8
    kw = dict(num_starts=2, fixing_sample_size=24, solving_sample_size=16, elite_threshold=0.2)
    for g1 in (0.05, 1e-7):
        sq = dict(sqa_slices=P, sqa_beta=3.0, sqa_gamma0=2.0, sqa_gamma1=g1)
        plan = spvar.Plan([gpu_problem(inst)], spvar.make_params(num_sweeps=T, sampler=spvar.SAMPLER_SQA, **sq, **kw))
        out = plan.run([44], device=False)
        plan.close()
        ref = O.solve(op, table(inst, T), 44, sampler=1, **sq, **kw)
        for s in range(2):
            for ph in range(ref.nphases[s]):
                c = ref.counts[s, ph]
                assert np.array_equal(np.asarray(out.energies[s, ph, :c]), ref.energies[s, ph, :c]), (g1, s, ph)


@pytest.mark.parametrize("kernel,block,shape", [("PM1", 256, "sqa-register"), ("GENERAL", 256, "sqa"),
                                                ("GENERAL", 512, "sqa")], ids=["si_register", "general_256",
                                                                              "general_512"])
@pytest.mark.parametrize("make,P", [(lambda: I.chimera_u10(3, 2132), 4), (lambda: I.chimera_u10(4, 2133), 8)],
                         ids=["u10_C3_P4", "u10_C4_P8"])
def test_solve_with_sqa_small_integer_couplers(cuda_lib, kernel, block, shape, make, P):
    """SQA on U_10 Chimera problems (couplers of ten magnitudes): the register
    form for small integer couplers and the general path, requested
    explicitly, are identical to the oracle in every phase."""
    from paper_1706_07826_gb300 import spvar
    inst = make()
    op = oracle_problem(inst)
    T, starts = 30, 2
    sq = dict(sqa_slices=P, sqa_beta=3.0, sqa_gamma0=2.5, sqa_gamma1=0.05)
    kw = dict(num_starts=starts, fixing_sample_size=24, solving_sample_size=16, elite_threshold=0.2)
    ref = O.solve(op, table(inst, T), 45, sampler=1, **sq, **kw)
    prm = spvar.make_params(num_sweeps=T, sampler=spvar.SAMPLER_SQA, replicas_per_block=4,
                            sweep_kernel=getattr(spvar, "SWEEP_" + kernel), sweep_block=block, **sq, **kw)
    plan = spvar.Plan([gpu_problem(inst)], prm)
    assert plan.shape()["kernel"] == shape
    out = plan.run([45], device=False)
    plan.close()
    for s in range(starts):
        for ph in range(ref.nphases[s]):
            c = ref.counts[s, ph]
            assert np.array_equal(np.asarray(out.energies[s, ph, :c]), ref.energies[s, ph, :c]), (s, ph)
        assert np.array_equal(np.asarray(out.best_state[s * inst.n:(s + 1) * inst.n]), ref.best_state[s])
