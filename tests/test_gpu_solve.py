"""GPU parity of Multi-start SPVAR (spvar_solve / plans, Alg. 2) against the
oracle: recorded energies, phase sizes, fix maps and best states are
identical in the batched (persistent + CUDA graph) and plain forms, for every
sweep shape, and for several problems of uneven size in one plan."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I

from gpu_cases import gpu_problem, oracle_problem, table, with_h

pytestmark = pytest.mark.gpu


def _oracle_solve(inst, T, seed, **kw):
    return O.solve(oracle_problem(inst), table(inst, T), seed, **kw)


def _check(out, ref, starts, P, n, slot0=0, fm0=0):
    for s in range(starts):
        g = slot0 + s
        assert int(out.nphases[g]) == ref.nphases[s]
        assert np.array_equal(np.asarray(out.counts[g]), ref.counts[s])
        assert np.array_equal(np.asarray(out.nfree[g]), ref.nfree[s])
        for ph in range(ref.nphases[s]):
            c = ref.counts[s, ph]
            assert np.array_equal(np.asarray(out.energies[g, ph, :c]), ref.energies[s, ph, :c]), (s, ph)
        assert int(out.best_energy[g]) == ref.best_e[s]
        a = fm0 + s * n
        assert np.array_equal(np.asarray(out.fixed[a:a + n]), ref.fixed[s])
        assert np.array_equal(np.asarray(out.best_state[a:a + n]), ref.best_state[s])


SCASES = [
    # name, instance, T, starts, S_fix, S_solve, elite, iterate, max_fix
    ("cubic_L4_ispvar", lambda: I.cubic3d(4, 1100), 120, 1, 256, 0, 0.1, True, 64),
    ("chimera_C4", lambda: I.chimera(4, 1200), 100, 3, 100, 100, 0.1, False, 1),
    ("weak_strong_C3", lambda: I.weak_strong(3, 1300), 80, 4, 40, 40, 0.2, False, 1),
    ("cubic_L5_odd_ispvar3", lambda: I.cubic3d(5, 1401), 60, 2, 64, 30, 0.2, True, 3),
    ("random_h", lambda: I.random_graph(30, 70, 3, jmax=3, hmax=2), 60, 3, 33, 19, 0.3, False, 1),
    # large problems: the persistence pass's CTAs own several 1024-spin count chunks and run
    # their 256-spin fold chunks in several rounds (odd L: more than two colour classes)
    ("cubic_L24_large", lambda: I.cubic3d(24, 1500), 12, 2, 16, 8, 0.25, False, 1),
    ("cubic_L31_odd_ispvar", lambda: I.cubic3d(31, 1501), 8, 1, 12, 8, 0.5, True, 2),
]


@pytest.mark.parametrize("form", [0, 1], ids=["batched", "plain"])
@pytest.mark.parametrize("name,make,T,starts,Sf,Ss,elite,iterate,mf", SCASES, ids=[c[0] for c in SCASES])
def test_solve_parity(cuda_lib, form, name, make, T, starts, Sf, Ss, elite, iterate, mf):
    from paper_1706_07826_gb300 import spvar
    inst = make()
    seed = 4242
    ref = _oracle_solve(inst, T, seed, num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss,
                        elite_threshold=elite, iterate=iterate, max_fix_phases=mf)
    prm = spvar.make_params(num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss, num_sweeps=T,
                            elite_threshold=elite, iterate=iterate, max_fix_phases=mf, form=form)
    out = spvar.solve(gpu_problem(inst), prm, seed)
    _check(out, ref, starts, mf + 1, inst.n)


SHAPES = [(4, 1, 256), (8, 1, 128), (32, 1, 512), (4, 2, 256), (8, 2, 128), (4, 2, 512), (16, 2, 256),
          (12, 2, 128), (4, 3, 256), (4, 3, 512), (4, 3, 1024), (8, 4, 0), (16, 4, 0), (32, 4, 0), (64, 4, 0),
          (4, 5, 128), (8, 5, 256), (32, 5, 512), (16, 5, 128)]


@pytest.mark.parametrize("rpb,kernel,block", SHAPES, ids=["%d-%d-%d" % s for s in SHAPES])
@pytest.mark.parametrize("make", [lambda: I.chimera(3, 9), lambda: I.cubic3d(5, 19)], ids=["chimera", "cubic_odd"])
def test_solve_identical_for_every_sweep_shape(cuda_lib, rpb, kernel, block, make):
    """General, register-resident, streaming, warp-per-quad and quad-group
    kernels, several replicas per CTA and block sizes (2 to 4 register slots
    per thread): all identical."""
    from paper_1706_07826_gb300 import spvar
    inst = make()
    T, seed = 50, 17
    ref = _oracle_solve(inst, T, seed, num_starts=2, fixing_sample_size=45, solving_sample_size=45,
                        elite_threshold=0.2)
    prm = spvar.make_params(num_starts=2, fixing_sample_size=45, solving_sample_size=45, num_sweeps=T,
                            elite_threshold=0.2, replicas_per_block=rpb, sweep_kernel=kernel, sweep_block=block)
    plan = spvar.Plan([gpu_problem(inst)], prm)
    want = {2: "pm1-register", 3: "pm1-streaming", 4: "pm1-warp", 5: "pm1-quads"}.get(kernel,
                                                                                     plan.shape()["kernel"])
    if kernel == 2 and block == 512 and inst.n == 125:
        want = "pm1-streaming"  # four colour classes need four slots; 512-thread CTAs have two
    assert plan.shape()["kernel"] == want
    _check(plan.run(seed, device=False), ref, 2, 2, inst.n)


def test_quad_group_kernel_uneven_problems(cuda_lib):
    """The quad-group kernel with problems of four sizes in one plan: its shared
    memory holds two quads of the largest, so smaller problems run more quads
    per work item (up to 15 here); all identical to the oracle."""
    from paper_1706_07826_gb300 import spvar
    insts = [I.cubic3d(L, 1500 + L) for L in (3, 6, 5, 4)]
    T, starts, Sf, Ss = 40, 2, 120, 60
    dmax = max(O.dmax(oracle_problem(i)) for i in insts)
    seeds = [21, 22, 23, 24]
    plan = spvar.Plan([gpu_problem(i) for i in insts],
                      spvar.make_params(num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss,
                                        num_sweeps=T, elite_threshold=0.1, replicas_per_block=8,
                                        sweep_kernel=spvar.SWEEP_PM1Q, sweep_block=128))
    assert plan.shape()["kernel"] == "pm1-quads"
    out = plan.run(seeds, device=False)
    plan.close()
    fm0 = 0
    for pi, inst in enumerate(insts):
        ref = O.solve(oracle_problem(inst), table(inst, T, dmax=dmax), seeds[pi], num_starts=starts,
                      fixing_sample_size=Sf, solving_sample_size=Ss, elite_threshold=0.1)
        _check(out, ref, starts, 2, inst.n, slot0=pi * starts, fm0=fm0)
        fm0 += starts * inst.n


def test_register_kernel_rejects_general_couplers(cuda_lib):
    """Couplers of several magnitudes at one spin have no register-kernel form."""
    from paper_1706_07826_gb300 import spvar
    prm = spvar.make_params(num_starts=1, fixing_sample_size=8, solving_sample_size=8, num_sweeps=4,
                            replicas_per_block=4, sweep_kernel=spvar.SWEEP_PM1)
    with pytest.raises(spvar.SpvarError):
        spvar.Plan([gpu_problem(I.random_graph(30, 60, 2, jmax=5, hmax=3))], prm)


UJ_SHAPES = [(4, 256), (8, 256), (16, 256), (4, 512), (4, 576), (8, 576), (4, 1024), (8, 1024)]


@pytest.mark.parametrize("rpb,block", UJ_SHAPES, ids=["%d-%d" % s for s in UJ_SHAPES])
@pytest.mark.parametrize("make", [lambda: I.weak_strong(2, 61), lambda: with_h(I.cubic3d(4, 62), 5, 20),
                                  lambda: I.chimera_u10(3, 63), lambda: I.chimera_u10(4, 64)],
                         ids=["weak_strong_x100", "pm1_big_h", "u10_C3", "u10_C4"])
def test_register_kernel_one_magnitude_per_spin(cuda_lib, rpb, block, make):
    """The register kernel's 16-bit-lane variants (one coupler magnitude per
    spin: weak-strong problems, +-1 problems with large biases; small integer
    couplers: U_10 Chimera problems): identical to the oracle for several
    launch shapes."""
    from paper_1706_07826_gb300 import spvar
    inst = make()
    T, seed = 50, 19
    ref = _oracle_solve(inst, T, seed, num_starts=2, fixing_sample_size=45, solving_sample_size=45,
                        elite_threshold=0.2)
    prm = spvar.make_params(num_starts=2, fixing_sample_size=45, solving_sample_size=45, num_sweeps=T,
                            elite_threshold=0.2, replicas_per_block=rpb, sweep_kernel=spvar.SWEEP_PM1,
                            sweep_block=block)
    plan = spvar.Plan([gpu_problem(inst)], prm)
    assert plan.shape()["kernel"] == "pm1-register"
    _check(plan.run([seed], device=False), ref, 2, 2, inst.n)
    plan.close()


def test_profiling_reports_sweep_time(cuda_lib):
    from paper_1706_07826_gb300 import spvar
    inst = I.chimera(4, 3)
    plan = spvar.Plan([gpu_problem(inst)], spvar.make_params(num_starts=2, fixing_sample_size=64,
                                                             solving_sample_size=32, num_sweeps=40))
    plan.set_profiling(True)
    plan.run(5, device=False)
    ms, n = plan.sweep_time()
    assert n == 2 and ms > 0 and plan.post_time() > 0


@pytest.mark.parametrize("iterate", [False, True], ids=["spvar", "ispvar"])
def test_loop_graph_equals_phase_by_phase(cuda_lib, iterate):
    """A batched run as one graph launch (device-side phase loop) gives the same
    results as phase-by-phase launches with the host in between (profiled)."""
    from paper_1706_07826_gb300 import spvar
    inst = I.cubic3d(4, 77)
    prm = spvar.make_params(num_starts=3, fixing_sample_size=48, solving_sample_size=0 if iterate else 24,
                            num_sweeps=30, elite_threshold=0.2, iterate=iterate, max_fix_phases=32 if iterate else 1)
    plan = spvar.Plan([gpu_problem(inst)], prm)
    a = plan.run(9, device=False)
    plan.set_profiling(True)
    b = plan.run(9, device=False)
    for f in ("energies", "counts", "nfree", "nphases", "fixed", "best_energy", "best_state"):
        assert np.array_equal(np.asarray(getattr(a, f)), np.asarray(getattr(b, f))), f
    ref = _oracle_solve(inst, 30, 9, num_starts=3, fixing_sample_size=48, solving_sample_size=0 if iterate else 24,
                        elite_threshold=0.2, iterate=iterate, max_fix_phases=32 if iterate else 1)
    _check(a, ref, 3, (32 if iterate else 1) + 1, inst.n)


def test_uneven_problems_in_one_plan(cuda_lib):
    """Problems of different sizes (3 colours for odd L) share one persistent launch per phase."""
    from paper_1706_07826_gb300 import spvar
    insts = [I.cubic3d(L, 1400 + L) for L in (3, 6, 5, 4)]
    T, starts, Sf, Ss = 60, 2, 48, 24
    dmax = max(O.dmax(oracle_problem(i)) for i in insts)
    seeds = [11, 12, 13, 14]
    plan = spvar.Plan([gpu_problem(i) for i in insts],
                      spvar.make_params(num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss,
                                        num_sweeps=T, elite_threshold=0.1))
    out = plan.run(seeds, device=False)
    fm0 = 0
    for pi, inst in enumerate(insts):
        ref = O.solve(oracle_problem(inst), table(inst, T, dmax=dmax), seeds[pi], num_starts=starts,
                      fixing_sample_size=Sf, solving_sample_size=Ss, elite_threshold=0.1)
        _check(out, ref, starts, 2, inst.n, slot0=pi * starts, fm0=fm0)
        fm0 += starts * inst.n
    # a second run of the same plan (graph replay) reproduces the first
    out2 = plan.run(seeds, device=False)
    assert np.array_equal(out2.energies, out.energies) or all(
        np.array_equal(out2.energies[s, p, :out.counts[s, p]], out.energies[s, p, :out.counts[s, p]])
        for s in range(len(insts) * starts) for p in range(2))
    attempts, phases = plan.stats()
    assert attempts == sum(int(out.counts[s, p]) * int(out.nfree[s, p]) * T
                           for s in range(len(insts) * starts) for p in range(2))


def test_chimera_c8_full_size_properties(cuda_lib):
    """The benchmark's workload (Chimera C8, 10 starts x (1000 + 1000) samples,
    1000 sweeps): phase-0 energies of sampled replicas match the oracle one by
    one, and every best state's recomputed energy is the reported best energy."""
    from paper_1706_07826_gb300 import spvar
    inst = I.chimera(8, 1200)
    T, seed, starts = 1000, 42, 10
    prm = spvar.make_params(num_starts=starts, fixing_sample_size=1000, solving_sample_size=1000,
                            num_sweeps=T, elite_threshold=0.1)
    out = spvar.solve(gpu_problem(inst), prm, seed)
    op = oracle_problem(inst)
    thr = table(inst, T)
    for st, r in ((0, 0), (3, 517), (9, 999)):
        _, e, _ = O.sample(op, thr, 1, seed, start=st, phase=0, r0=r)
        assert out.energies[st, 0, r] == e[0]
    for st in range(starts):
        assert out.best_energy[st] == O.energy(op, out.best_state[st * inst.n:(st + 1) * inst.n])
        assert out.best_energy[st] == min(out.energies[st, 0].min(), out.energies[st, 1].min())
        assert out.nfree[st, 1] == inst.n - int((out.fixed[st * inst.n:(st + 1) * inst.n] != 0).sum())


def test_start_offset_shards_reproduce_full_run(cuda_lib):
    """Two plans over start blocks [0, 3) and [3, 5) equal one plan over [0, 5)."""
    from paper_1706_07826_gb300 import spvar
    inst = I.chimera(3, 41)
    kw = dict(fixing_sample_size=40, solving_sample_size=20, num_sweeps=40, elite_threshold=0.2)
    full = spvar.solve(gpu_problem(inst), spvar.make_params(num_starts=5, **kw), 99)
    a = spvar.solve(gpu_problem(inst), spvar.make_params(num_starts=3, start_offset=0, **kw), 99)
    b = spvar.solve(gpu_problem(inst), spvar.make_params(num_starts=2, start_offset=3, **kw), 99)
    assert np.array_equal(np.concatenate([a.best_energy, b.best_energy]), full.best_energy)
    assert np.array_equal(np.concatenate([a.fixed, b.fixed]), full.fixed)


BCASES = [
    ("cubic_L4_tau34", lambda: I.cubic3d(4, 31), 40, 3, 64, 40, 0.1, (3, 4)),
    ("chimera_C4_tau910", lambda: I.chimera(4, 33), 60, 2, 100, 64, 0.1, (9, 10)),
    ("random_h", lambda: I.random_graph(40, 60, 5, jmax=3, hmax=2), 50, 3, 48, 33, 0.2, (1, 1)),
    ("random_5_components", lambda: I.random_graph(60, 70, 9, jmax=3, hmax=1), 40, 3, 64, 40, 0.2, (3, 4)),
]


@pytest.mark.parametrize("form", [0, 1], ids=["batched", "plain"])
@pytest.mark.parametrize("name,make,T,starts,Sf,Ss,elite,tau", BCASES, ids=[c[0] for c in BCASES])
def test_component_boost_parity(cuda_lib, form, name, make, T, starts, Sf, Ss, elite, tau):
    """Sec. II.C boosting of the solving sample: identical to the oracle."""
    from paper_1706_07826_gb300 import spvar
    inst = make()
    ref = _oracle_solve(inst, T, 8, num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss,
                        elite_threshold=elite, fix_num=tau[0], fix_den=tau[1], boost=True)
    prm = spvar.make_params(num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss, num_sweeps=T,
                            elite_threshold=elite, fix_num=tau[0], fix_den=tau[1], form=form, component_boost=True)
    _check(spvar.solve(gpu_problem(inst), prm, 8), ref, starts, 2, inst.n)


TCASES = [
    ("random_trees", lambda: I.random_graph(40, 48, 17, jmax=3, hmax=2), 60, 3, 32, 24, 0.2, (1, 1), False, 1),
    ("random_zero_bias", lambda: (lambda x: (setattr(x, "h", np.zeros(x.n, np.int32)), x)[1])(
        I.random_graph(50, 60, 23, jmax=2, hmax=0)), 50, 2, 40, 20, 0.25, (1, 1), False, 1),
    ("random_5_components_boost", lambda: I.random_graph(60, 70, 9, jmax=3, hmax=1), 40, 3, 64, 40, 0.2, (3, 4),
     True, 1),
    ("cubic_L4_ispvar_tree", lambda: I.cubic3d(4, 32), 60, 2, 64, 0, 0.1, (3, 4), False, 64),
]


@pytest.mark.parametrize("form", [0, 1], ids=["batched", "plain"])
@pytest.mark.parametrize("name,make,T,starts,Sf,Ss,elite,tau,boost,mf", TCASES, ids=[c[0] for c in TCASES])
def test_tree_preprocess_parity(cuda_lib, form, name, make, T, starts, Sf, Ss, elite, tau, boost, mf):
    """Sec. II.C tree pre-processing after SPVAR reductions: identical to the oracle
    (fix maps, recorded energies, best states with inferred spins restored)."""
    from paper_1706_07826_gb300 import spvar
    inst = make()
    iterate = mf > 1
    ref = _oracle_solve(inst, T, 6, num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss,
                        elite_threshold=elite, fix_num=tau[0], fix_den=tau[1], boost=boost, tree=True,
                        iterate=iterate, max_fix_phases=mf)
    prm = spvar.make_params(num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss, num_sweeps=T,
                            elite_threshold=elite, fix_num=tau[0], fix_den=tau[1], form=form,
                            component_boost=boost, tree_preprocess=True, iterate=iterate, max_fix_phases=mf)
    _check(spvar.solve(gpu_problem(inst), prm, 6), ref, starts, mf + 1, inst.n)


CCASES = [
    # name, instance, T, starts, S_corr, corr_elite, S_fix, S_solve, elite, iterate, max_fix, tree, boost
    ("chimera_C4_paper_split", lambda: I.chimera(4, 41), 80, 3, 80, 0.2, 60, 60, 0.2, False, 1, False, False),
    ("cubic_L4_corr", lambda: I.cubic3d(4, 42), 60, 2, 64, 0.3, 48, 48, 0.2, False, 1, False, False),
    ("cubic_L5_odd_corr_ispvar", lambda: I.cubic3d(5, 43), 50, 2, 40, 0.25, 32, 16, 0.2, True, 4, False, False),
    ("random_zero_bias_tree_boost", lambda: I.random_graph(50, 60, 23, jmax=2, hmax=0), 50, 2, 40, 0.3, 30, 24,
     0.25, False, 1, True, True),
    ("random_h_skipped", lambda: I.random_graph(30, 70, 3, jmax=3, hmax=2), 40, 2, 50, 0.3, 33, 19, 0.3, False, 1,
     False, False),
]


@pytest.mark.parametrize("form", [0, 1], ids=["batched", "plain"])
@pytest.mark.parametrize("name,make,T,starts,Sc,ce,Sf,Ss,elite,iterate,mf,tree,boost", CCASES,
                         ids=[c[0] for c in CCASES])
def test_correlation_fixing_parity(cuda_lib, form, name, make, T, starts, Sc, ce, Sf, Ss, elite, iterate, mf, tree,
                                   boost):
    """Sec. II.C correlation fixing of zero-bias problems (its own phase, sample
    size and elite threshold; skipped with bias): identical to the oracle."""
    from paper_1706_07826_gb300 import spvar
    inst = make()
    ref = _oracle_solve(inst, T, 12, num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss,
                        elite_threshold=elite, iterate=iterate, max_fix_phases=mf, tree=tree, boost=boost,
                        corr_sample_size=Sc, corr_elite_threshold=ce)
    prm = spvar.make_params(num_starts=starts, fixing_sample_size=Sf, solving_sample_size=Ss, num_sweeps=T,
                            elite_threshold=elite, iterate=iterate, max_fix_phases=mf, form=form,
                            tree_preprocess=tree, component_boost=boost, corr_sample_size=Sc,
                            corr_elite_threshold=ce)
    out = spvar.solve(gpu_problem(inst), prm, 12)
    _check(out, ref, starts, mf + 2, inst.n)
    if not inst.h.any():
        assert all(int(out.counts[s][0]) == Sc for s in range(starts))


def test_correlation_fixing_rejects_bad_parameters(cuda_lib):
    from paper_1706_07826_gb300 import spvar
    gp = gpu_problem(I.chimera(2, 3))
    for kw in (dict(corr_sample_size=-1), dict(corr_sample_size=8, corr_num=2, corr_den=1),
               dict(corr_sample_size=8, corr_elite_threshold=0.0)):
        with pytest.raises(spvar.SpvarError):
            spvar.solve(gp, spvar.make_params(num_starts=1, fixing_sample_size=8, solving_sample_size=8,
                                              num_sweeps=10, **kw), 1)


CHUNK_CASES = [
    # name, instance, T, sweeps per launch, replicas_per_block, kernel, block, extra oracle/plan options
    ("register", lambda: I.chimera(3, 41), 60, 25, 8, 2, 128, {}),
    ("quads_odd", lambda: I.cubic3d(5, 42), 50, 7, 8, 5, 256, {}),
    ("streaming", lambda: I.cubic3d(5, 43), 40, 13, 4, 3, 256, {}),
    ("warp", lambda: I.chimera(3, 44), 40, 16, 8, 4, 0, {}),
    ("general_h", lambda: I.random_graph(30, 70, 3, jmax=3, hmax=2), 45, 20, 4, 1, 256, {}),
    ("weak_strong_16bit", lambda: I.weak_strong(3, 45), 48, 17, 4, 2, 256, {}),
    ("autotuned_ispvar", lambda: I.cubic3d(4, 46), 60, 11, 0, 0, 0, dict(iterate=True, max_fix_phases=64)),
    ("boost_tree", lambda: I.random_graph(40, 48, 17, jmax=3, hmax=2), 36, 9, 0, 0, 0, dict(boost=True, tree=True)),
]


@pytest.mark.parametrize("form", [0, 1], ids=["batched", "plain"])
@pytest.mark.parametrize("name,make,T,spl,rpb,kernel,block,opts", CHUNK_CASES, ids=[c[0] for c in CHUNK_CASES])
def test_phase_in_several_sweep_launches(cuda_lib, form, name, make, T, spl, rpb, kernel, block, opts):
    """A phase annealed over ceil(T / sweeps_per_launch) launches, each resuming
    from the states the previous one wrote, equals the oracle (every random word
    is keyed by the absolute sweep), for every sweep kernel, ISPVAR, boosting and
    tree pre-processing."""
    from paper_1706_07826_gb300 import spvar
    inst = make()
    seed, starts = 99, 3
    iterate = opts.get("iterate", False)
    mf = opts.get("max_fix_phases", 1)
    Ss = 0 if iterate else 30
    ref = _oracle_solve(inst, T, seed, num_starts=starts, fixing_sample_size=40, solving_sample_size=Ss,
                        elite_threshold=0.2, iterate=iterate, max_fix_phases=mf, boost=opts.get("boost", False),
                        tree=opts.get("tree", False))
    prm = spvar.make_params(num_starts=starts, fixing_sample_size=40, solving_sample_size=Ss, num_sweeps=T,
                            elite_threshold=0.2, iterate=iterate, max_fix_phases=mf, form=form,
                            replicas_per_block=rpb, sweep_kernel=kernel, sweep_block=block,
                            component_boost=opts.get("boost", False), tree_preprocess=opts.get("tree", False),
                            sweeps_per_launch=spl)
    plan = spvar.Plan([gpu_problem(inst)], prm)
    assert plan.shape()["sweeps_per_launch"] == spl
    out = plan.run(seed, device=False)
    plan.close()
    _check(out, ref, starts, mf + 1, inst.n)


def test_sweeps_per_launch_rejected_with_sqa(cuda_lib):
    from paper_1706_07826_gb300 import spvar
    prm = spvar.make_params(num_starts=1, fixing_sample_size=8, solving_sample_size=8, num_sweeps=10,
                            sampler=spvar.SAMPLER_SQA, sqa_slices=4, sweeps_per_launch=5)
    with pytest.raises(spvar.SpvarError) as e:
        spvar.Plan([gpu_problem(I.chimera(2, 1))], prm)
    assert e.value.code == spvar.EINVAL


def test_solve_keeps_and_rebinds_its_plan(cuda_lib):
    """spvar_solve keeps its plan for problems of the same structure: problems
    with the same graph but other couplers, solved in turn (and a problem of
    another structure in between), each give the oracle's result; so do
    solves after the kept plans are released."""
    from paper_1706_07826_gb300 import spvar
    T, seed = 40, 77
    kw = dict(num_starts=2, fixing_sample_size=48, solving_sample_size=24, elite_threshold=0.2)
    prm = spvar.make_params(num_sweeps=T, **kw)
    same = [I.chimera(4, 1201), I.chimera(4, 1202), I.chimera(4, 1203)]
    other = I.cubic3d(5, 1204)
    refs = {id(x): _oracle_solve(x, T, seed, **kw) for x in same + [other]}
    spvar.solve_cache_release()
    for x in same + [other] + same[::-1]:
        out = spvar.solve(gpu_problem(x), prm, seed)
        _check(out, refs[id(x)], 2, 2, x.n)
    spvar.solve_cache_release()
    out = spvar.solve(gpu_problem(same[1]), prm, seed)
    _check(out, refs[id(same[1])], 2, 2, same[1].n)
    spvar.solve_cache_release()


def test_solve_from_several_threads(cuda_lib):
    """Concurrent spvar_solve calls on problems of one structure: each call
    takes a kept plan for itself (or builds one), results as the oracle's."""
    import threading
    from paper_1706_07826_gb300 import spvar
    T, seed = 30, 91
    kw = dict(num_starts=2, fixing_sample_size=40, solving_sample_size=20, elite_threshold=0.2)
    prm = spvar.make_params(num_sweeps=T, **kw)
    insts = [I.chimera(3, 1300 + i) for i in range(6)]
    refs = [_oracle_solve(x, T, seed, **kw) for x in insts]
    probs = [gpu_problem(x) for x in insts]
    outs = [None] * len(insts)
    errs = []

    def work(i):
        try:
            for _ in range(3):
                outs[i] = spvar.solve(probs[i], prm, seed)
        except Exception as e:  # reported below
            errs.append(e)

    th = [threading.Thread(target=work, args=(i,)) for i in range(len(insts))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for i, x in enumerate(insts):
        _check(outs[i], refs[i], 2, 2, x.n)
    spvar.solve_cache_release()


LARGE_ELITE_CASES = [
    # name, instance, T, S_fix, S_solve, elite: every case has k > 512, where the elite's
    # candidates (at least k) exceed the rank placement's 512 and the full sort runs
    # inside the persistence pass
    ("ferromagnet_C2_ties", lambda: _ferromagnet(I.chimera(2, 1601)), 80, 1500, 300, 0.6),
    ("random_16_S8192", lambda: I.random_graph(16, 30, 1602, jmax=2, hmax=1), 30, 8192, 64, 0.1),
    ("random_8_S16384_max", lambda: I.random_graph(8, 12, 1603, jmax=2, hmax=0), 20, 16384, 32, 0.1),
]


def _ferromagnet(inst):
    inst.J = -np.ones_like(inst.J)
    return inst


@pytest.mark.parametrize("name,make,T,Sf,Ss,elite", LARGE_ELITE_CASES, ids=[c[0] for c in LARGE_ELITE_CASES])
def test_persistence_pass_with_large_elites(cuda_lib, name, make, T, Sf, Ss, elite):
    """The fused persistence pass with elites larger than 512 samples (heavily
    tied energies; sample counts up to the library's maximum, the pass's
    largest shared-memory layout): identical to the oracle."""
    from paper_1706_07826_gb300 import spvar
    inst = make()
    seed = 5150
    kw = dict(num_starts=2, fixing_sample_size=Sf, solving_sample_size=Ss, elite_threshold=elite)
    ref = _oracle_solve(inst, T, seed, **kw)
    out = spvar.solve(gpu_problem(inst), spvar.make_params(num_sweeps=T, **kw), seed)
    _check(out, ref, 2, 2, inst.n)
