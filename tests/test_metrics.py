"""Success metrics (Sec. III.A) against their closed forms."""
import math

import numpy as np

from paper_1706_07826_gb300 import metrics as M


def test_fraction_gap_residual():
    best = [-100, -98, -50, 0]
    known = [-100, -100, -50, 0]
    assert M.fraction_solved(best, known) == 0.75
    assert list(M.gap(best, known)) == [0, 2, 0, 0]
    r = M.residual(best, known)
    assert r[0] == 0 and r[2] == 0 and r[3] == 0
    assert abs(r[1] - 2.0) < 1e-12  # 100 * 2 / 100


def test_starts99_closed_forms():
    assert M.starts99(0.0) is None
    assert M.starts99(1.0) == 1.0
    assert abs(M.starts99(0.5) - math.log(0.01) / math.log(0.5)) < 1e-12
    # p = 1 - 0.01^(1/k) needs exactly k starts
    for k in (2, 5, 17):
        assert abs(M.starts99(1 - 0.01 ** (1 / k)) - k) < 1e-9


def test_r99_spvar_is_starts_times_sample_size():
    flags = [True, False, False, True]  # p = 0.5
    assert abs(M.r99_spvar(flags, 1000) - 1000 * math.log(0.01) / math.log(0.5)) < 1e-9
    assert M.r99_spvar([False] * 3, 1000) is None
    assert M.r99_spvar([True] * 3, 500) == 500


def test_bootstrap_median():
    assert M.bootstrap_median_r99([7.0] * 9, resamples=50) == 7.0
    assert M.bootstrap_median_r99([None, None]) is None
    vals = [1.0, 2.0, 3.0, None, 100.0]
    a = M.bootstrap_median_r99(vals, resamples=200, seed=3)
    b = M.bootstrap_median_r99(vals, resamples=200, seed=3)
    assert a == b and 1.0 <= a <= 100.0
    # the median of the measurable values when nothing is resampled away
    g = np.random.default_rng(5)
    big = list(g.integers(1, 1000, 401).astype(float))
    assert abs(M.bootstrap_median_r99(big, resamples=300) - np.median(big)) < 0.15 * np.median(big)


def _table2():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_parameters.txt")
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        name, elite, corr_elite, starts, total, sweeps = [c.strip() for c in line.split("|")]
        lo, _, hi = total.partition("-")
        rows.append(dict(name=name, elite=float(elite), corr_elite=None if corr_elite == "-" else float(corr_elite),
                         starts=int(starts), totals=sorted({int(lo), int(hi or lo)}),
                         sweeps=[int(x) for x in sweeps.split(",")]))
    return rows


def test_sample_split_of_the_paper_parameters():
    """The appendix's split of Table II's total sample sizes: half and half
    with bias; 40 % for the correlation step and the rest halved without."""
    rows = _table2()
    assert len(rows) == 6
    seen = set()
    for r in rows:
        for total in r["totals"]:
            c, f, s = M.sample_split(total, zero_bias=False)
            assert (c, f, s) == (0, total // 2, total - total // 2) and f == s
            c, f, s = M.sample_split(total, zero_bias=True)
            assert c + f + s == total and abs(c - 0.4 * total) < 1 and f == s
            seen.add((total, c, f))
    # the sizes the paper's sets used: 100, 500 and 1000 samples per start
    assert (500, 200, 150) in seen and (1000, 400, 300) in seen and (100, 40, 30) in seen
    assert M.sample_split(7, True) == (2, 2, 3) and M.sample_split(7, False) == (0, 3, 4)

