"""Oracle pins for the problem layer (Sec. I): CSR construction, colour
classes of the sweep order, dmax and the energy.  References are scipy/numpy
routines and closed forms, never the oracle itself."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse import csgraph

from oracle import oracle as O
from paper_1706_07826_gb300 import instances as I


def _csr(inst):
    return O.csr_from_edges(inst.n, inst.ei, inst.ej, inst.J, inst.h, inst.offset, inst.scale)


def _dense_upper(inst):
    M = np.zeros((inst.n, inst.n), np.int64)
    for a, b, j in zip(inst.ei, inst.ej, inst.J):
        M[min(a, b), max(a, b)] += j
    return M


INSTANCES = [I.cubic3d(3, 1), I.cubic3d(4, 2), I.cubic3d(5, 3), I.chimera(2, 4), I.chimera(8, 1200),
             I.weak_strong(3, 5), I.random_graph(12, 30, 6), I.random_graph(1, 0, 7)]


@pytest.mark.parametrize("inst", INSTANCES, ids=lambda x: x.name)
def test_csr_matches_scipy(inst):
    p = _csr(inst)
    rows = np.concatenate([inst.ei, inst.ej])
    cols = np.concatenate([inst.ej, inst.ei])
    vals = np.concatenate([inst.J, inst.J])
    ref = sp.csr_matrix((vals, (rows, cols)), shape=(inst.n, inst.n))
    ref.sort_indices()
    assert np.array_equal(p.row_ptr, ref.indptr)
    assert np.array_equal(p.col, ref.indices)
    assert np.array_equal(p.val, ref.data)


def test_csr_rejects_bad_edges():
    with pytest.raises(ValueError):
        O.csr_from_edges(3, [0], [0], [1], [0, 0, 0])          # self loop
    with pytest.raises(ValueError):
        O.csr_from_edges(3, [0, 1], [1, 0], [1, 1], [0, 0, 0])  # repeated pair
    with pytest.raises(ValueError):
        O.csr_from_edges(3, [0], [3], [1], [0, 0, 0])          # out of range


def test_generator_shapes():
    c = I.cubic3d(6, 1)
    assert c.n == 216 and c.m == 3 * 216
    assert len({(min(a, b), max(a, b)) for a, b in zip(c.ei, c.ej)}) == c.m
    assert np.all(np.bincount(np.concatenate([c.ei, c.ej])) == 6)
    ch = I.chimera(8, 1)
    assert ch.n == 512 and ch.m == 1472
    assert np.bincount(np.concatenate([ch.ei, ch.ej])).max() == 6
    ws = I.weak_strong(12, 1)
    assert ws.n == 1152 and ws.scale == 100
    assert set(np.unique(ws.h)) == {-100, 44}
    assert set(np.unique(ws.J)) == {-100, 100}


@pytest.mark.parametrize("inst", INSTANCES, ids=lambda x: x.name)
def test_colour_classes(inst):
    p = _csr(inst)
    colour, ncol = O.colour(p)
    if p.n == 0:
        return
    assert colour.min() == 0 and colour.max() == ncol - 1
    # valid: no coupler inside a class
    for i in range(p.n):
        for q in range(p.row_ptr[i], p.row_ptr[i + 1]):
            assert colour[i] != colour[p.col[q]]
    A = sp.csr_matrix((np.ones(p.nnz), p.col, p.row_ptr), shape=(p.n, p.n))
    ncomp, labels = csgraph.connected_components(A, directed=False)
    # bipartite test by scipy's BFS distances from each component's lowest index
    parity = np.full(p.n, -1)
    for c in range(ncomp):
        root = int(np.flatnonzero(labels == c)[0])
        d = csgraph.shortest_path(A, unweighted=True, indices=root)
        members = labels == c
        parity[members] = (d[members].astype(int) % 2)
    bip = all(parity[i] != parity[p.col[q]] for i in range(p.n) for q in range(p.row_ptr[i], p.row_ptr[i + 1]))
    if bip:
        assert np.array_equal(colour, parity)
    else:
        # first-fit: each colour is the smallest one no lower-index neighbour has
        for i in range(p.n):
            lower = {colour[p.col[q]] for q in range(p.row_ptr[i], p.row_ptr[i + 1]) if p.col[q] < i}
            assert colour[i] == min(set(range(len(lower) + 1)) - lower)


def test_colour_counts_of_paper_graphs():
    assert O.colour(_csr(I.cubic3d(4, 1)))[1] == 2
    assert O.colour(_csr(I.cubic3d(6, 1)))[1] == 2
    assert O.colour(_csr(I.chimera(8, 1)))[1] == 2
    assert O.colour(_csr(I.cubic3d(5, 1)))[1] >= 3   # odd periodic L is not bipartite
    assert O.colour(_csr(I.cubic3d(7, 1)))[1] >= 3


@pytest.mark.parametrize("inst", INSTANCES, ids=lambda x: x.name)
def test_dmax(inst):
    p = _csr(inst)
    s = np.abs(inst.h).astype(np.int64)
    np.add.at(s, inst.ei, np.abs(inst.J))
    np.add.at(s, inst.ej, np.abs(inst.J))
    assert O.dmax(p) == 2 * int(s.max(initial=0))


@pytest.mark.parametrize("inst", INSTANCES, ids=lambda x: x.name)
def test_energy_matches_dense_quadratic_form(inst):
    p = _csr(inst)
    M = _dense_upper(inst)
    g = np.random.default_rng(3)
    for _ in range(20):
        s = (g.integers(0, 2, inst.n) * 2 - 1).astype(np.int8)
        ref = int(s.astype(np.int64) @ M @ s.astype(np.int64) + inst.h.astype(np.int64) @ s)
        assert O.energy(p, s) == ref


def test_ferromagnet_ground_energy_closed_form():
    inst = I.cubic3d(4, 1)
    inst.J[:] = -1
    p = _csr(inst)
    assert O.energy(p, np.ones(inst.n, np.int8)) == -3 * inst.n
    assert O.energy(p, -np.ones(inst.n, np.int8)) == -3 * inst.n
