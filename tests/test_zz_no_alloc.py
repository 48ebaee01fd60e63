"""The allocation-free reduction (spvar_reduce_noalloc).

Some callers cannot call cudaMalloc while they run -- code inside a fully
committed device-memory budget, or a runtime that owns all device
allocations -- so this entry point keeps its working arrays in a static
device array and writes into buffers the caller allocated beforehand.  Its
output must equal the allocating spvar_reduce exactly, call after call (the
static array keeps the previous call's contents).  This file is collected
last so that a failure here never hides another test's result.
"""
import numpy as np
import pytest

from paper_1706_07826_gb300 import instances as I

pytestmark = pytest.mark.gpu


def _noalloc(spvar, torch, gp, fixed_t, n, nnz):
    dev = dict(dtype=torch.int32, device="cuda")
    out = dict(row_ptr=torch.full((n + 1,), -7, **dev), col=torch.full((max(nnz, 1),), -7, **dev),
               val=torch.full((max(nnz, 1),), -7, **dev), h=torch.full((max(n, 1),), -7, **dev),
               offset=torch.zeros(1, dtype=torch.int64, device="cuda"),
               old_of_new=torch.full((max(n, 1),), -7, **dev), n_out=torch.zeros(1, **dev))
    spvar.reduce_noalloc(gp, fixed_t, out["row_ptr"], out["col"], out["val"], out["h"], out["offset"],
                         out["old_of_new"], out["n_out"])
    torch.cuda.synchronize()
    m = int(out["n_out"].item())
    rp = out["row_ptr"][:m + 1].cpu().numpy()
    return dict(n=m, row_ptr=rp, col=out["col"][:rp[-1]].cpu().numpy(), val=out["val"][:rp[-1]].cpu().numpy(),
                h=out["h"][:m].cpu().numpy(), offset=int(out["offset"].item()),
                old_of_new=out["old_of_new"][:m].cpu().numpy())


@pytest.mark.parametrize("make", [lambda: I.weak_strong(4, 31), lambda: I.cubic3d(7, 32)], ids=["weak_strong", "cubic"])
def test_noalloc_reduce_matches_spvar_reduce_twice(cuda_lib, make):
    import torch
    spvar = cuda_lib
    inst = make()
    inst.offset = 123
    gp = spvar.Problem.from_instance(inst)
    info = gp.info()
    g = np.random.default_rng(3)
    # two calls in a row with different fixings: the second must not see the first's scratch
    for fixed in (g.choice([-1, 0, 0, 1], inst.n), g.choice([-1, 0, 1, 1, 0], inst.n)):
        fixed_t = torch.from_numpy(fixed.astype(np.int8)).cuda()
        ref, ref_oon = spvar.reduce(gp, fixed_t)
        want = ref.download()
        got = _noalloc(spvar, torch, gp, fixed_t, info.n, info.nnz)
        assert got["n"] == want["n"]
        for k in ("row_ptr", "col", "val", "h"):
            assert np.array_equal(got[k], want[k]), k
        assert got["offset"] == want["offset"]
        assert np.array_equal(got["old_of_new"], ref_oon.cpu().numpy())


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
