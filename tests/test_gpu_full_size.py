"""GPU parity at the benchmark's full sizes, in the launch configuration that
bench.py times (autotuned batched plans): the oracle recomputes sampled
replicas one by one, or a whole start where that takes seconds.

- weak-strong Chimera C12 x100 (N = 1152), 32 starts x (250 + 250) samples,
  1000 sweeps: one whole start (both phases, fix map, best state) and sampled
  phase-0 replicas of other starts;
- the uneven batch of 64 3D +-J problems (L 6..12), 2000 + 2000 samples,
  1000 sweeps, one persistent launch per phase for all of them: one whole
  start of an L = 6 problem and sampled phase-0 replicas of the largest and
  of odd-L (three-colour) problems;
- SQA on Chimera C8 (N = 512), 16 slices, 10 starts x (500 + 500) runs, 1000
  sweeps: sampled phase-0 runs (recorded energies);
- reduced-degeneracy Chimera C8 with biases (U_10, Sec. III.C): one whole
  start and sampled replicas;
- PTICM (Sec. III.D) on 3D +-J L = 10, 304 runs x 32 temperatures x 2
  replicas, 1000 sweeps: two whole runs (kept lists, final states).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I

from gpu_cases import gpu_problem, oracle_problem, table

pytestmark = pytest.mark.gpu


def test_c3_weak_strong_full_size(cuda_lib):
    from paper_1706_07826_gb300 import spvar
    inst = I.weak_strong(12, 1300)
    T, seed, starts = 1000, 2, 32
    kw = dict(fixing_sample_size=250, solving_sample_size=250, elite_threshold=0.2)
    plan = spvar.Plan([gpu_problem(inst)], spvar.make_params(num_starts=starts, num_sweeps=T, **kw))
    out = plan.run(seed, device=False)
    plan.close()
    op = oracle_problem(inst)
    thr = table(inst, T)
    # one whole start, both phases
    st = 17
    ref = O.solve(op, thr, seed, num_starts=1, start0=st, **kw)
    assert int(out.nphases[st]) == ref.nphases[0]
    for ph in range(ref.nphases[0]):
        c = ref.counts[0, ph]
        assert np.array_equal(np.asarray(out.energies[st, ph, :c]), ref.energies[0, ph, :c]), ph
    n = inst.n
    assert np.array_equal(np.asarray(out.fixed[st * n:(st + 1) * n]), ref.fixed[0])
    assert np.array_equal(np.asarray(out.best_state[st * n:(st + 1) * n]), ref.best_state[0])
    # sampled phase-0 replicas of other starts
    for s, r in ((0, 0), (9, 131), (31, 249)):
        _, e, _ = O.sample(op, thr, 1, seed, start=s, phase=0, r0=r)
        assert out.energies[s, 0, r] == e[0] + inst.offset


def test_c4_uneven_batch_full_size(cuda_lib):
    from paper_1706_07826_gb300 import spvar
    insts = I.uneven_batch(64, 6, 12, seed=1400)
    T = 1000
    kw = dict(fixing_sample_size=2000, solving_sample_size=2000, elite_threshold=0.1)
    plan = spvar.Plan([gpu_problem(x) for x in insts], spvar.make_params(num_starts=1, num_sweeps=T, **kw))
    seeds = [1401 + i for i in range(len(insts))]
    out = plan.run(seeds, device=False)
    plan.close()
    Ls = [round(x.n ** (1 / 3)) for x in insts]
    # one whole start of the first L = 6 problem (its slot is its index: one start per problem)
    i6 = Ls.index(6)
    inst = insts[i6]
    ref = O.solve(oracle_problem(inst), table(inst, T), seeds[i6], num_starts=1, **kw)
    assert int(out.nphases[i6]) == ref.nphases[0]
    for ph in range(ref.nphases[0]):
        c = ref.counts[0, ph]
        assert np.array_equal(np.asarray(out.energies[i6, ph, :c]), ref.energies[0, ph, :c]), ph
    fm0 = sum(x.n for x in insts[:i6])
    assert np.array_equal(np.asarray(out.best_state[fm0:fm0 + inst.n]), ref.best_state[0])
    # sampled phase-0 replicas of the largest problem and of odd-L problems
    picks = [Ls.index(12), Ls.index(11), Ls.index(7)]
    for i, r in zip(picks, (0, 1234, 1999)):
        inst = insts[i]
        _, e, _ = O.sample(oracle_problem(inst), table(inst, T), 1, seeds[i], start=0, phase=0, r0=r)
        assert out.energies[i, 0, r] == e[0] + inst.offset, (Ls[i], r)


def test_sqa_chimera_c8_full_size(cuda_lib):
    from paper_1706_07826_gb300 import spvar
    inst = I.chimera(8, 1100)
    T, P, seed, starts = 1000, 16, 2300, 10
    prm = spvar.make_params(num_starts=starts, fixing_sample_size=500, solving_sample_size=500, num_sweeps=T,
                            elite_threshold=0.1, sampler=spvar.SAMPLER_SQA, sqa_slices=P, sqa_beta=3.0,
                            sqa_gamma0=3.0, sqa_gamma1=0.01)
    plan = spvar.Plan([gpu_problem(inst)], prm)
    out = plan.run([seed], device=False)
    plan.close()
    op = oracle_problem(inst)
    ent = O.sqa_table(T, P, 3.0, O.gamma_linear(T, 3.0, 0.01), O.dmax(op), 1)
    for st, r in ((0, 0), (4, 311), (9, 499)):
        _, e, _ = O.sqa_sample(op, ent, P, 1, seed, start=st, phase=0, r0=r)
        assert out.energies[st, 0, r] == e[0] + inst.offset, (st, r)


def test_u10_chimera_c8_small_integer_couplers(cuda_lib):
    """Reduced-degeneracy Chimera C8 with biases (the U_10 class of Sec. III.C:
    couplers of ten magnitudes, the register kernel's small-integer variant):
    an autotuned plan of 4 starts x (100 + 100) samples at 1000 sweeps equals
    the oracle on one whole start; sampled phase-0 replicas of the others match
    one by one."""
    from paper_1706_07826_gb300 import spvar
    inst = I.chimera_u10(8, 2500)
    T, seed, starts = 1000, 8, 4
    kw = dict(fixing_sample_size=100, solving_sample_size=100, elite_threshold=0.1)
    plan = spvar.Plan([gpu_problem(inst)], spvar.make_params(num_starts=starts, num_sweeps=T, **kw))
    out = plan.run(seed, device=False)
    plan.close()
    op = oracle_problem(inst)
    thr = table(inst, T)
    st = 2
    ref = O.solve(op, thr, seed, num_starts=1, start0=st, **kw)
    for ph in range(ref.nphases[0]):
        c = ref.counts[0, ph]
        assert np.array_equal(np.asarray(out.energies[st, ph, :c]), ref.energies[0, ph, :c]), ph
    n = inst.n
    assert np.array_equal(np.asarray(out.best_state[st * n:(st + 1) * n]), ref.best_state[0])
    for s, r in ((0, 0), (1, 57), (3, 99)):
        _, e, _ = O.sample(op, thr, 1, seed, start=s, phase=0, r0=r)
        assert out.energies[s, 0, r] == e[0] + inst.offset, (s, r)


def test_sqa_u10_chimera_c8_full_size(cuda_lib):
    """SQA on a U_10 Chimera C8 problem with biases (16 slices, 1000 sweeps,
    10 starts x (500 + 500) runs, autotuned): sampled phase-0 runs match the
    oracle one by one."""
    from paper_1706_07826_gb300 import spvar
    inst = I.chimera_u10(8, 2500)
    T, P, seed, starts = 1000, 16, 2400, 10
    prm = spvar.make_params(num_starts=starts, fixing_sample_size=500, solving_sample_size=500, num_sweeps=T,
                            elite_threshold=0.1, sampler=spvar.SAMPLER_SQA, sqa_slices=P, sqa_beta=3.0,
                            sqa_gamma0=3.0, sqa_gamma1=0.01)
    plan = spvar.Plan([gpu_problem(inst)], prm)
    out = plan.run([seed], device=False)
    plan.close()
    op = oracle_problem(inst)
    ent = O.sqa_table(T, P, 3.0, O.gamma_linear(T, 3.0, 0.01), O.dmax(op), inst.scale)
    for st, r in ((0, 0), (5, 250), (9, 499)):
        _, e, _ = O.sqa_sample(op, ent, P, 1, seed, start=st, phase=0, r0=r)
        assert out.energies[st, 0, r] == e[0] + inst.offset, (st, r)


def test_pticm_3d_l10_full_size(cuda_lib):
    """The PTICM benchmark launch (304 runs, 32 temperatures geometric 0.2 ->
    3.0, cluster moves and kept lists in the lower half, 1000 sweeps): the
    first and the last run equal the oracle bit for bit."""
    import torch
    from paper_1706_07826_gb300 import spvar
    inst = I.cubic3d(10, 1600)
    betas = np.geomspace(0.2, 3.0, 32)
    T, runs = 1000, 304
    g = spvar.pticm_sample(gpu_problem(inst), betas, T, spvar.energy_range(inst), K=10, num_runs=runs, seed=4)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in g.items()}
    op = oracle_problem(inst)
    for run in (0, runs - 1):
        ref = O.pticm_sample(op, betas, T, K=10, seed=4, start=run)
        assert np.array_equal(g["nkept"][run], ref["nkept"]), run
        for q, nk in enumerate(ref["nkept"]):
            assert np.array_equal(g["kept_e"][run, q, :nk], ref["kept_e"][q, :nk] + inst.offset), (run, q)
            assert np.array_equal(spvar.unpack_spins(g["kept"][run, q, :nk], inst.n), ref["kept"][q, :nk]), (run, q)
        assert np.array_equal(spvar.unpack_spins(g["final_states"][run], inst.n), ref["final"]), run
        assert np.array_equal(g["final_e"][run], ref["final_e"] + inst.offset), run
