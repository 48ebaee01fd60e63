"""GPU parity of the third sampler, PTICM (parallel tempering with
isoenergetic cluster moves, Sec. III.D; spvar_pticm_sample), against the
oracle: every run's kept lists (states, energies, counts) and every replica's
final state and energy identical, bit for bit, for +-1, integer and U_10
couplers, odd and even temperature counts, and with exchanges or cluster
moves switched off; and Alg. 2 with PTICM as the sampler of every phase (one
run per start and phase, the kept lists as the sample) in plans, batched and
plain, against the oracle's Alg. 2."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I

from gpu_cases import gpu_problem, oracle_problem, table, with_h

pytestmark = pytest.mark.gpu

CASES = [
    # name, instance, betas, sweeps, runs, options
    ("random_h_R6", lambda: I.random_graph(20, 40, 3, jmax=3, hmax=2), np.geomspace(0.2, 2.5, 6), 40, 3, {}),
    ("chimera_C3_R8", lambda: I.chimera(3, 2140), np.geomspace(0.2, 3.0, 8), 30, 2, {}),
    ("cubic_L4_R4", lambda: I.cubic3d(4, 2141), np.geomspace(0.3, 3.0, 4), 30, 2, {}),
    ("cubic_L5_odd_h_R5", lambda: with_h(I.cubic3d(5, 2143), 6, 2), np.geomspace(0.3, 2.0, 5), 25, 2, {}),
    ("u10_C3_R8", lambda: I.chimera_u10(3, 2142), np.geomspace(0.2, 3.0, 8), 30, 2, {}),
    ("no_exchange", lambda: I.random_graph(16, 30, 7, jmax=2, hmax=1), np.geomspace(0.3, 2.0, 4), 30, 2,
     dict(exchange=False)),
    ("no_icm_keep_all", lambda: I.chimera(2, 2144), np.geomspace(0.3, 2.0, 6), 30, 2,
     dict(icm=False, keep_from=0)),
    ("icm_all_keep_top", lambda: I.random_graph(18, 36, 9, jmax=3, hmax=2), np.geomspace(0.2, 2.5, 6), 30, 1,
     dict(icm_from=0, keep_from=5)),
    ("one_temperature", lambda: I.random_graph(12, 20, 11, jmax=2, hmax=2), np.array([1.3]), 40, 2, {}),
    # at least as many replica quads as warps: each warp owns whole quads for a sweep
    ("chimera_C3_R16", lambda: I.chimera(3, 2145), np.geomspace(0.2, 3.0, 16), 20, 2, {}),
    ("random_h_R19_uneven_quads", lambda: I.random_graph(24, 50, 13, jmax=3, hmax=2), np.geomspace(0.2, 3.0, 19),
     20, 2, {}),
]


@pytest.mark.parametrize("name,make,betas,T,runs,opt", CASES, ids=[c[0] for c in CASES])
def test_pticm_parity(cuda_lib, name, make, betas, T, runs, opt):
    import torch
    from paper_1706_07826_gb300 import spvar
    inst = make()
    op = oracle_problem(inst)
    g = spvar.pticm_sample(gpu_problem(inst), betas, T, spvar.energy_range(inst), K=10, num_runs=runs, seed=77,
                           start0=5, phase=1, **opt)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in g.items()}
    for run in range(runs):
        ref = O.pticm_sample(op, betas, T, K=10, seed=77, start=5 + run, phase=1, **opt)
        assert np.array_equal(g["nkept"][run], ref["nkept"]), run
        for q, nk in enumerate(ref["nkept"]):
            assert np.array_equal(g["kept_e"][run, q, :nk], ref["kept_e"][q, :nk] + inst.offset), (run, q)
            states = spvar.unpack_spins(g["kept"][run, q, :nk], inst.n)
            assert np.array_equal(states, ref["kept"][q, :nk]), (run, q)
        assert np.array_equal(spvar.unpack_spins(g["final_states"][run], inst.n), ref["final"]), run
        assert np.array_equal(g["final_e"][run], ref["final_e"] + inst.offset), run


def test_pticm_limits(cuda_lib):
    from paper_1706_07826_gb300 import spvar
    small = I.random_graph(10, 15, 1, jmax=2, hmax=1)
    gp = gpu_problem(small)
    with pytest.raises(spvar.SpvarError):
        spvar.pticm_sample(gp, np.geomspace(0.1, 3.0, 65), 2, spvar.energy_range(small))   # more than 64 temperatures
    big = I.cubic3d(13, 3)  # N = 2197 > 2048
    with pytest.raises(spvar.SpvarError):
        spvar.pticm_sample(gpu_problem(big), np.geomspace(0.1, 3.0, 4), 2, spvar.energy_range(big))
    mid = I.cubic3d(12, 5)  # N = 1728: 64 temperatures of replicas and queues need more than one CTA's shared memory
    with pytest.raises(spvar.SpvarError):
        spvar.pticm_sample(gpu_problem(mid), np.geomspace(0.1, 3.0, 64), 2, spvar.energy_range(mid))


PT_CASES = [
    # name, instance, T, R, K, starts, iterate, max_fix, tree
    ("cubic_L3", lambda: I.cubic3d(3, 5), 30, 6, 4, 2, False, 1, False),
    ("chimera_C2_h", lambda: with_h(I.chimera(2, 6), 7, 2), 24, 8, 3, 3, False, 1, False),
    ("cubic_L4_ispvar_tree", lambda: I.cubic3d(4, 8), 20, 6, 3, 2, True, 40, True),
    ("random_odd_colours", lambda: I.random_graph(40, 90, 12, jmax=2, hmax=1), 25, 5, 5, 2, False, 1, False),
]


@pytest.mark.parametrize("form", [0, 1], ids=["batched", "plain"])
@pytest.mark.parametrize("name,make,T,R,K,starts,iterate,mf,tree", PT_CASES, ids=[c[0] for c in PT_CASES])
def test_solve_with_pticm_sampler_matches_oracle(cuda_lib, form, name, make, T, R, K, starts, iterate, mf, tree):
    """Alg. 2 with PTICM (Sec. III.D) as the sampler of every phase: each
    phase's sample is the run's kept lists; recorded energies, sample sizes,
    free spins, fix maps and best states equal the oracle's."""
    from paper_1706_07826_gb300 import spvar
    from test_gpu_solve import _check
    inst = make()
    S = spvar.pticm_sample_size(R, K)
    Ss = 0 if iterate else S
    seed = 31
    ref = O.solve(oracle_problem(inst), table(inst, T), seed, num_starts=starts, fixing_sample_size=S,
                  solving_sample_size=Ss, elite_threshold=0.25, iterate=iterate, max_fix_phases=mf, tree=tree,
                  sampler=2, pticm_temps=R, pticm_keep=K, pticm_beta0=0.3, pticm_beta1=2.5)
    prm = spvar.make_params(num_starts=starts, fixing_sample_size=S, solving_sample_size=Ss, num_sweeps=T,
                            elite_threshold=0.25, iterate=iterate, max_fix_phases=mf, tree_preprocess=tree, form=form,
                            sampler=spvar.SAMPLER_PTICM, pticm_temps=R, pticm_keep=K, pticm_beta0=0.3, pticm_beta1=2.5)
    plan = spvar.Plan([gpu_problem(inst)], prm)
    out = plan.run(seed, device=False)
    att, _ = plan.stats()
    plan.close()
    _check(out, ref, starts, mf + 1, inst.n)
    assert att > 0


def test_pticm_sampler_parameters_are_checked(cuda_lib):
    from paper_1706_07826_gb300 import spvar
    inst = I.cubic3d(3, 2)
    bad = [dict(fixing_sample_size=10, solving_sample_size=10),        # not 2 (R - R/2) K
           dict(fixing_sample_size=24, solving_sample_size=24, component_boost=True),
           dict(fixing_sample_size=24, solving_sample_size=24, num_sweeps=0)]
    for kw in bad:
        kw.setdefault("num_sweeps", 10)
        with pytest.raises(spvar.SpvarError) as e:
            spvar.Plan([gpu_problem(inst)], spvar.make_params(sampler=spvar.SAMPLER_PTICM, pticm_temps=6,
                                                               pticm_keep=4, **kw))
        assert e.value.code == spvar.EINVAL
    big = I.cubic3d(13, 3)  # 2197 spins > 2048
    with pytest.raises(spvar.SpvarError) as e:
        spvar.Plan([gpu_problem(big)], spvar.make_params(sampler=spvar.SAMPLER_PTICM, pticm_temps=6, pticm_keep=4,
                                                         fixing_sample_size=24, solving_sample_size=24,
                                                         num_sweeps=10))
    assert e.value.code == spvar.ELIMIT


def test_pticm_sampler_with_problems_of_different_size(cuda_lib):
    """Two problems of different size and colouring in one PTICM plan (one run
    per start of each, in one launch per phase): each equals the oracle."""
    from paper_1706_07826_gb300 import spvar
    from test_gpu_solve import _check
    insts = [I.cubic3d(4, 21), I.chimera(2, 22)]
    T, R, K, starts = 20, 6, 3, 2
    S = spvar.pticm_sample_size(R, K)
    prm = spvar.make_params(num_starts=starts, fixing_sample_size=S, solving_sample_size=S, num_sweeps=T,
                            elite_threshold=0.25, sampler=spvar.SAMPLER_PTICM, pticm_temps=R, pticm_keep=K,
                            pticm_beta0=0.3, pticm_beta1=2.5)
    plan = spvar.Plan([gpu_problem(x) for x in insts], prm)
    seeds = [41, 42]
    out = plan.run(seeds, device=False)
    plan.close()
    fm0 = 0
    for pi, inst in enumerate(insts):
        ref = O.solve(oracle_problem(inst), table(inst, T), seeds[pi], num_starts=starts, fixing_sample_size=S,
                      solving_sample_size=S, elite_threshold=0.25, sampler=2, pticm_temps=R, pticm_keep=K,
                      pticm_beta0=0.3, pticm_beta1=2.5)
        _check(out, ref, starts, 2, inst.n, slot0=pi * starts, fm0=fm0)
        fm0 += starts * inst.n
