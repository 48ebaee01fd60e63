"""Success metrics of Multi-start SPVAR (Sec. III.A), host side.

- fraction of problems solved: the best energy found equals the best known one;
- gap: best found - best known;
- residual: 100 (best found - best known) / |best known|, in percent;
- R99: the sample size needed to observe the best known energy with 99 %
  confidence.  For Multi-start SPVAR the per-start success rate p gives the
  number of starts ln(0.01) / ln(1 - p) (one start when p = 1, not measurable
  when p = 0), multiplied by the total sample size of one start;
- the figures report the mean over 1000 bootstrap resamples of the problems of
  the median of the measurable R99 values (Sec. III.C).

Also the split of a start's total sample between the steps of Alg. 2 that
the paper's benchmarking used (appendix, Table II).
"""
import math

import numpy as np


def fraction_solved(best, known):
    """Fraction of problems whose best energy reaches the best known energy."""
    best, known = np.asarray(best), np.asarray(known)
    return float(np.mean(best <= known)) if best.size else float("nan")


def gap(best, known):
    """best - known per problem (0 when solved)."""
    return np.asarray(best, np.int64) - np.asarray(known, np.int64)


def residual(best, known):
    """Relative gap in percent: 100 (best - known) / |known| (0 where known is 0 and solved)."""
    best = np.asarray(best, np.float64)
    known = np.asarray(known, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = 100.0 * (best - known) / np.abs(known)
    return np.where(best == known, 0.0, r)


def starts99(p):
    """Starts needed to see the best known energy with 99 % confidence at a
    per-start success rate p; None when p = 0 (not measurable)."""
    if p <= 0:
        return None
    if p >= 1:
        return 1.0
    return math.log(0.01) / math.log(1.0 - p)


def r99_spvar(start_success, samples_per_start):
    """R99 of one problem from its per-start success flags (Sec. III.A): the
    mean success rate gives starts99, times the total sample size of a start."""
    s = starts99(float(np.mean(np.asarray(start_success, bool)))) if len(start_success) else None
    return None if s is None else s * samples_per_start


def bootstrap_median_r99(r99s, resamples=1000, seed=0):
    """Mean over bootstrap resamples of the problems of the median of the
    measurable R99 values (None entries are not measurable and are dropped
    from each resample).  Returns None if no resample has a measurable value."""
    vals = list(r99s)
    if not vals:
        return None
    g = np.random.default_rng(seed)
    meds = []
    for _ in range(resamples):
        pick = [vals[i] for i in g.integers(0, len(vals), len(vals))]
        m = [v for v in pick if v is not None]
        if m:
            meds.append(float(np.median(m)))
    return float(np.mean(meds)) if meds else None


def sample_split(total, zero_bias):
    """(correlation, fixing, solving) sample sizes of one start whose total
    sample is `total` (appendix, Table II): for problems with bias, half for
    the SPVAR fixing step and half for solving; for zero-bias problems 40 % for
    the correlation pre-fixing step and the rest divided equally between
    fixing and solving.  Where the shares are not whole, the correlation step
    takes 40 % rounded down and the solving step the odd sample left over."""
    if total < 0:
        raise ValueError("total sample size must be >= 0")
    corr = (2 * total) // 5 if zero_bias else 0
    rest = total - corr
    fixing = rest // 2
    return corr, fixing, rest - fixing
