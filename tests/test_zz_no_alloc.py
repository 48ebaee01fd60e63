"""The allocation-free reduction (spvar_reduce_noalloc).

Some callers cannot call cudaMalloc while they run -- code inside a fully
committed device-memory budget, or a runtime that owns all device
allocations -- so this entry point keeps its working arrays in a static
device array and writes into buffers the caller allocated beforehand.  Its
output must equal the oracle's reduction (Alg. 1, update of J and h) and the
allocating spvar_reduce exactly, call after call (the static array keeps the
previous call's contents), on original and already reduced problems, with
nothing, something or everything fixed, on the default and on an explicit
stream.  This file is collected last so that a failure here never hides
another test's result.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I

from gpu_cases import empty, oracle_problem

pytestmark = pytest.mark.gpu


def _noalloc(spvar, torch, gp, fixed_t, n, nnz, stream=None):
    dev = dict(dtype=torch.int32, device="cuda")
    out = dict(row_ptr=torch.full((n + 1,), -7, **dev), col=torch.full((max(nnz, 1),), -7, **dev),
               val=torch.full((max(nnz, 1),), -7, **dev), h=torch.full((max(n, 1),), -7, **dev),
               offset=torch.zeros(1, dtype=torch.int64, device="cuda"),
               old_of_new=torch.full((max(n, 1),), -7, **dev), n_out=torch.full((1,), -7, **dev))
    spvar.reduce_noalloc(gp, fixed_t, out["row_ptr"], out["col"], out["val"], out["h"], out["offset"],
                         out["old_of_new"], out["n_out"], stream=stream)
    torch.cuda.synchronize()
    m = int(out["n_out"].item())
    rp = out["row_ptr"][:m + 1].cpu().numpy()
    return dict(n=m, row_ptr=rp, col=out["col"][:rp[-1]].cpu().numpy(), val=out["val"][:rp[-1]].cpu().numpy(),
                h=out["h"][:m].cpu().numpy(), offset=int(out["offset"].item()),
                old_of_new=out["old_of_new"][:m].cpu().numpy())


def _check(spvar, torch, gp, op, colours, fixed, stream=None):
    """noalloc output == oracle reduction == spvar_reduce; returns the oracle's
    reduced problem and colours for a second level."""
    info = gp.info()
    fixed_t = torch.from_numpy(fixed.astype(np.int8)).cuda() if info.n else torch.zeros(1, dtype=torch.int8,
                                                                                         device="cuda")
    got = _noalloc(spvar, torch, gp, fixed_t, info.n, info.nnz, stream)
    red, col2, oon = O.reduce(op, fixed, colours)
    assert got["n"] == red.n
    assert np.array_equal(got["row_ptr"], red.row_ptr)
    assert np.array_equal(got["col"], red.col) and np.array_equal(got["val"], red.val)
    assert np.array_equal(got["h"], red.h)
    assert got["offset"] == red.offset
    assert np.array_equal(got["old_of_new"], oon)
    ref, ref_oon = spvar.reduce(gp, fixed_t)
    want = ref.download()
    assert got["n"] == want["n"]
    for k in ("row_ptr", "col", "val", "h"):
        assert np.array_equal(got[k], want[k]), k
    assert got["offset"] == ref.info().offset
    assert np.array_equal(got["old_of_new"], ref_oon.cpu().numpy())
    return ref, red, col2


CASES = [
    ("weak_strong", lambda: I.weak_strong(4, 31)),
    ("cubic_odd", lambda: I.cubic3d(7, 32)),
    ("chimera", lambda: I.chimera(5, 33)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_noalloc_reduce_matches_oracle_twice(cuda_lib, name, make):
    """Two calls in a row with different fixings, then none and all fixed: the
    later calls must not see the earlier calls' scratch contents."""
    import torch
    spvar = cuda_lib
    inst = make()
    inst.offset = 123
    gp = spvar.Problem.from_instance(inst)
    op = oracle_problem(inst)
    colours = O.colour(op)
    g = np.random.default_rng(3)
    for fixed in (g.choice([-1, 0, 0, 1], inst.n), g.choice([-1, 0, 1, 1, 0], inst.n),
                  np.zeros(inst.n, np.int8), g.choice([-1, 1], inst.n)):
        _check(spvar, torch, gp, op, colours, fixed.astype(np.int8))


def test_noalloc_reduce_of_a_reduced_problem_on_a_stream(cuda_lib):
    """A second-level reduction (the input is spvar_reduce's output, whose
    capacities exceed its size) on an explicit non-default stream."""
    import torch
    spvar = cuda_lib
    inst = I.cubic3d(8, 34)
    inst.h = np.random.default_rng(5).integers(-2, 3, inst.n).astype(np.int32)
    gp = spvar.Problem.from_instance(inst)
    op = oracle_problem(inst)
    g = np.random.default_rng(6)
    f1 = g.choice([-1, 0, 0, 0, 1], inst.n).astype(np.int8)
    gp2, red, col2 = _check(spvar, torch, gp, op, O.colour(op), f1)
    assert gp2.info().n == red.n and red.n < inst.n
    f2 = g.choice([-1, 0, 0, 1], red.n).astype(np.int8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _check(spvar, torch, gp2, red, col2, f2, stream=s)
    _check(spvar, torch, gp2, red, col2, f2[::-1].copy())


def test_noalloc_reduce_of_an_empty_problem(cuda_lib):
    import torch
    spvar = cuda_lib
    inst = empty()
    gp = spvar.Problem.from_instance(inst)
    got = _noalloc(spvar, torch, gp, torch.zeros(1, dtype=torch.int8, device="cuda"), 0, 0)
    assert got["n"] == 0 and list(got["row_ptr"]) == [0] and got["offset"] == inst.offset


def test_noalloc_reduce_rejects_sizes_beyond_its_static_array(cuda_lib):
    import torch
    spvar = cuda_lib
    inst = I.cubic3d(26, 5)  # 17576 spins > 16384
    gp = spvar.Problem.from_instance(inst)
    n, nnz = gp.info().n, gp.info().nnz
    z = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(spvar.SpvarError) as e:
        spvar.reduce_noalloc(gp, torch.zeros(n, dtype=torch.int8, device="cuda"), z,
                             torch.zeros(nnz, dtype=torch.int32, device="cuda"),
                             torch.zeros(nnz, dtype=torch.int32, device="cuda"), z, torch.zeros(1, dtype=torch.int64,
                             device="cuda"), z, z)
    assert e.value.code == spvar.ELIMIT
