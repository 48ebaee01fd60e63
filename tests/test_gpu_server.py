"""GPU tests of the continuous-batching request loop (spvar_server_*).

Each request's result must be identical whether it ran alone (spvar_solve)
or inside a mix of requests of different sizes that arrive while others are
in flight and wait for device memory; one small request is also checked
against the oracle directly."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I

from gpu_cases import gpu_problem, oracle_problem, table

pytestmark = pytest.mark.gpu

KW = dict(num_starts=3, fixing_sample_size=48, solving_sample_size=24, num_sweeps=60, elite_threshold=0.2)


def _alone(spvar, inst, seed):
    return spvar.solve(gpu_problem(inst), spvar.make_params(**KW), seed)


def _same(a, b):
    assert np.array_equal(a.best_energy, b.best_energy)
    assert np.array_equal(a.fixed, b.fixed)
    assert np.array_equal(a.best_state, b.best_state)
    assert np.array_equal(a.counts, b.counts)
    assert np.array_equal(a.nfree, b.nfree)
    for s in range(a.counts.shape[0]):
        for p in range(a.counts.shape[1]):
            c = a.counts[s, p]
            assert np.array_equal(a.energies[s, p, :c], b.energies[s, p, :c])


def _server(spvar, budget, max_requests=3, pm1=False, sweeps_per_step=0, kernel=None):
    prm = spvar.make_params(**KW, sweep_kernel=(kernel if kernel is not None else spvar.SWEEP_PM1) if pm1 else 0)
    return spvar.Server(prm, budget, max_n=1000, max_nnz=6000, max_degree=6, max_dmax=12, max_requests=max_requests,
                        sweeps_per_step=sweeps_per_step)


SERVER_CASES = [("general", False, 0, None), ("pm1", True, 0, None), ("pm1_steps17", True, 17, None),
                ("general_steps25", False, 25, None), ("pm1_streaming_steps9", True, 9, 3),
                ("pm1_quads", True, 0, 5), ("pm1_quads_steps13", True, 13, 5)]


@pytest.mark.parametrize("name,pm1,sps,kernel", SERVER_CASES, ids=[c[0] for c in SERVER_CASES])
def test_results_identical_alone_and_in_the_mix(cuda_lib, name, pm1, sps, kernel):
    """Requests of mixed sizes that arrive while others are in flight and wait
    for device memory: each result equals the request solved alone, whole
    phases or sweep chunks per engine step, on the quad-group, streaming and
    general kernels."""
    spvar = cuda_lib
    insts = [I.cubic3d(4, 61), I.chimera(4, 62), I.cubic3d(5, 63), I.cubic3d(6, 64), I.chimera(3, 65)]
    seeds = [101, 102, 103, 104, 105]
    # budget for about two of these requests at a time: the rest queue for memory
    srv = _server(spvar, budget=600 << 10, pm1=pm1, sweeps_per_step=sps, kernel=kernel)
    ids = [srv.submit(insts[0], seeds[0])]
    srv.step()                                   # request 0 runs its first phase alone
    ids += [srv.submit(insts[i], seeds[i]) for i in (1, 2, 3)]
    saw_queue = srv.stats()["queued"] > 0
    srv.step()
    ids.append(srv.submit(insts[4], seeds[4]))
    steps = 0
    while srv.step() > 0 or srv.stats()["queued"] > 0:
        saw_queue |= srv.stats()["queued"] > 0
        steps += 1
        assert steps < 1000
    for rid, inst, seed in zip(ids, insts, seeds):
        info = srv.info(rid)
        assert info.state == 2 and info.latency_s > 0
        _same(srv.result(rid), _alone(spvar, inst, seed))
    assert saw_queue
    assert srv.stats()["done"] == len(ids)
    srv.close()


@pytest.mark.parametrize("pm1,sps", [(False, 0), (True, 7)], ids=["general", "pm1_steps7"])
def test_server_request_matches_oracle(cuda_lib, pm1, sps):
    spvar = cuda_lib
    inst = I.cubic3d(3, 70)
    srv = _server(spvar, budget=4 << 20, pm1=pm1, sweeps_per_step=sps)
    rid = srv.submit(inst, 7)
    while srv.step() > 0:
        pass
    out = srv.result(rid)
    ref = O.solve(oracle_problem(inst), table(inst, KW["num_sweeps"], dmax=12), 7, num_starts=3,
                  fixing_sample_size=48, solving_sample_size=24, elite_threshold=0.2)
    assert np.array_equal(out.best_energy, ref.best_e)
    assert np.array_equal(out.fixed.reshape(3, -1), ref.fixed)
    srv.close()


def test_background_engine_thread(cuda_lib):
    spvar = cuda_lib
    insts = [I.cubic3d(4, 80 + i) for i in range(4)]
    srv = _server(spvar, budget=32 << 20, max_requests=2)
    srv.start()
    ids = [srv.submit(inst, 200 + i) for i, inst in enumerate(insts)]
    for rid in ids:
        assert srv.info(rid, timeout=60.0).state == 2
    srv.stop()
    for i, (rid, inst) in enumerate(zip(ids, insts)):
        _same(srv.result(rid), _alone(spvar, inst, 200 + i))
        srv.release(rid)
    srv.close()


def test_server_limits(cuda_lib):
    spvar = cuda_lib
    srv = _server(spvar, budget=256 << 10)
    with pytest.raises(spvar.SpvarError) as e:
        srv.submit(I.cubic3d(11, 1), 1)          # 1331 spins > max_n
    assert e.value.code == spvar.ELIMIT
    with pytest.raises(spvar.SpvarError) as e:
        srv.submit(I.cubic3d(9, 1), 1)           # fits max_n but never fits the 256 KB budget
    assert e.value.code == spvar.EBUDGET
    with pytest.raises(spvar.SpvarError):
        srv.submit(I.weak_strong(2, 1), 1)       # dmax beyond the table
    srv.close()


def test_server_sweep_time_counts_every_step(cuda_lib):
    spvar = cuda_lib
    srv = _server(spvar, budget=8 << 20, pm1=True, sweeps_per_step=20)
    srv.submit(I.cubic3d(4, 90), 3)
    steps = 0
    while srv.step() > 0:
        steps += 1
    ms, n = srv.sweep_time()
    assert n == steps + 1 and ms > 0
    srv.close()


@pytest.mark.parametrize("pm1", [False, True], ids=["general", "pm1"])
def test_sqa_requests_identical_alone_and_in_the_mix(cuda_lib, pm1):
    """The second sampler in the request loop: requests sampled by SQA (4
    Trotter slices) give in a mix exactly what each gives solved alone, and one
    request equals the oracle's Alg. 2 with SQA in every phase."""
    spvar = cuda_lib
    sqa = dict(sampler=spvar.SAMPLER_SQA, sqa_slices=4, sqa_beta=2.0, sqa_gamma0=2.5, sqa_gamma1=0.05)
    prm = spvar.make_params(**KW, **sqa, sweep_kernel=spvar.SWEEP_PM1 if pm1 else 0)
    srv = spvar.Server(prm, 600 << 10, max_n=400, max_nnz=3000, max_degree=6, max_dmax=12, max_requests=3)
    insts = [I.cubic3d(4, 161), I.chimera(3, 162), I.cubic3d(5, 163), I.chimera(2, 164)]
    ids = [srv.submit(insts[0], 11)]
    srv.step()
    ids += [srv.submit(x, 12 + i) for i, x in enumerate(insts[1:])]
    steps = 0
    while srv.step() > 0 or srv.stats()["queued"] > 0:
        steps += 1
        assert steps < 100
    for rid, inst, seed in zip(ids, insts, [11, 12, 13, 14]):
        alone = spvar.solve(gpu_problem(inst), spvar.make_params(**KW, **sqa), seed)
        _same(srv.result(rid), alone)
    inst = insts[1]
    op = oracle_problem(inst)
    ref = O.solve(op, table(inst, KW["num_sweeps"], dmax=12), 12, num_starts=3, fixing_sample_size=48,
                  solving_sample_size=24, elite_threshold=0.2, sampler=1, sqa_slices=4, sqa_beta=2.0, sqa_gamma0=2.5,
                  sqa_gamma1=0.05)
    out = srv.result(ids[1])
    assert np.array_equal(out.best_energy, ref.best_e)
    assert np.array_equal(out.fixed.reshape(3, -1), ref.fixed)
    srv.close()


def test_sqa_server_rejects_sweep_steps(cuda_lib):
    spvar = cuda_lib
    prm = spvar.make_params(**KW, sampler=spvar.SAMPLER_SQA, sqa_slices=4)
    with pytest.raises(spvar.SpvarError) as e:
        spvar.Server(prm, 1 << 20, max_n=100, max_nnz=600, max_degree=6, max_dmax=12, sweeps_per_step=10)
    assert e.value.code == spvar.EINVAL
