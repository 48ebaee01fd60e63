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
  replicas, 1000 sweeps: two whole runs (kept lists, final states);
- ISPVAR on 3D +-J L = 4 (N = 64), 256 samples, 1000 sweeps, phases until
  every spin is fixed: every phase's energies, the fix map and the best state;
- the served stream through spvar_server_* (3D +-J, L = 20, 13 and 8 in one
  mix, 20 starts x (250 + 250) samples, 5000 sweeps in 500-sweep engine
  steps, elite 0.2, the server sized for N = 8000): one whole start of the L = 8 request and sampled
  phase-0 replicas of the L = 20 and odd-L requests.
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


def test_c1_cubic_l4_ispvar_full_size(cuda_lib):
    """ISPVAR (Sec. II.B) on a 3D +-J L = 4 problem at its benchmark sizes:
    one start, 256 samples per phase, 1000 sweeps, elite 0.1, SPVAR phases
    until every spin is fixed (autotuned batched plan, one graph launch)."""
    from paper_1706_07826_gb300 import spvar
    inst = I.cubic3d(4, 1100)
    T, seed = 1000, 2
    kw = dict(fixing_sample_size=256, solving_sample_size=0, elite_threshold=0.1, iterate=True, max_fix_phases=64)
    plan = spvar.Plan([gpu_problem(inst)], spvar.make_params(num_starts=1, num_sweeps=T, **kw))
    out = plan.run(seed, device=False)
    plan.close()
    ref = O.solve(oracle_problem(inst), table(inst, T), seed, num_starts=1, **kw)
    assert ref.nphases[0] > 2
    assert int(out.nphases[0]) == ref.nphases[0]
    assert np.array_equal(np.asarray(out.counts[0]), ref.counts[0])
    assert np.array_equal(np.asarray(out.nfree[0]), ref.nfree[0])
    for ph in range(ref.nphases[0]):
        c = ref.counts[0, ph]
        assert np.array_equal(np.asarray(out.energies[0, ph, :c]), ref.energies[0, ph, :c]), ph
    assert int(out.best_energy[0]) == ref.best_e[0]
    assert np.array_equal(np.asarray(out.fixed[:inst.n]), ref.fixed[0])
    assert np.all(ref.fixed[0] != 0)  # run to exhaustion: every spin fixed
    assert np.array_equal(np.asarray(out.best_state[:inst.n]), ref.best_state[0])


def test_c5_served_stream_full_size(cuda_lib):
    """The served stream at its benchmark sizes: three 3D +-J requests
    (L = 20, N = 8000; odd L = 13, three colour classes; L = 8) in one mix
    through the continuous-batching server configured as the benchmark runs it
    (N <= 8000, 20 starts x (250 + 250) samples, 5000 sweeps in 500-sweep
    engine steps, elite 0.2, quad-group kernel).  The
    oracle recomputes one whole start of the L = 8 request and sampled
    phase-0 replicas (first, middle, last) of the other two."""
    from paper_1706_07826_gb300 import spvar
    T, starts = 5000, 20
    kw = dict(fixing_sample_size=250, solving_sample_size=250, elite_threshold=0.2)
    prm = spvar.make_params(num_starts=starts, num_sweeps=T, sweep_kernel=spvar.SWEEP_PM1, **kw)
    srv = spvar.Server(prm, 8 << 30, max_n=8000, max_nnz=48000, max_degree=6, max_dmax=12, max_requests=32,
                       sweeps_per_step=500)
    insts = {20: I.cubic3d(20, 1520), 13: I.cubic3d(13, 1513), 8: I.cubic3d(8, 1508)}
    seeds = {20: 1620, 13: 1613, 8: 1608}
    ids = {}
    ids[20] = srv.submit(insts[20], seeds[20])
    srv.step()                                   # the L = 20 request runs 500 sweeps alone, the others join
    ids[13] = srv.submit(insts[13], seeds[13])
    ids[8] = srv.submit(insts[8], seeds[8])
    steps = 0
    while srv.step() > 0 or srv.stats()["queued"] > 0:
        steps += 1
        assert steps < 1000
    out = {L: srv.result(ids[L]) for L in ids}
    srv.close()
    # one whole start of the L = 8 request
    inst = insts[8]
    op = oracle_problem(inst)
    thr = table(inst, T, dmax=12)
    st = 11
    ref = O.solve(op, thr, seeds[8], num_starts=1, start0=st, **kw)
    o = out[8]
    assert np.array_equal(o.counts[st], ref.counts[0]) and np.array_equal(o.nfree[st], ref.nfree[0])
    for ph in range(ref.nphases[0]):
        c = ref.counts[0, ph]
        assert np.array_equal(o.energies[st, ph, :c], ref.energies[0, ph, :c]), ph
    assert int(o.best_energy[st]) == ref.best_e[0]
    n = inst.n
    assert np.array_equal(o.fixed[st * n:(st + 1) * n], ref.fixed[0])
    assert np.array_equal(o.best_state[st * n:(st + 1) * n], ref.best_state[0])
    # sampled phase-0 replicas of the largest and of the odd-L request
    for L, picks in ((20, ((0, 0), (10, 124), (19, 249))), (13, ((0, 0), (7, 125), (19, 249)))):
        inst = insts[L]
        op = oracle_problem(inst)
        thr = table(inst, T, dmax=12)
        for s, r in picks:
            _, e, _ = O.sample(op, thr, 1, seeds[L], start=s, phase=0, r0=r)
            assert out[L].energies[s, 0, r] == e[0] + inst.offset, (L, s, r)
