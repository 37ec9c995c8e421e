"""Monte Carlo standard error of a pooled log Z_hat, for the whole-run checks.

R independent runs (different seeds, or further rounds of one run, which redraw every
particle) give log Z_hat_r with delta-method standard errors se_r = sqrt(1/ESS_r - 1/N).  The
check compares the mean of the log Z_hat_r with the reference value within 3 standard errors
of that mean, taking the larger of two estimates of it: the delta method, sqrt(sum se_r^2) / R,
and the replicate spread, std_r(log Z_hat_r) / sqrt(R).  The spread guards against heavy-tailed
weights, for which the delta method is optimistic; log Z_hat's own bias (about -se^2 / 2 by
Jensen's inequality) is far below the bar at the sizes used.
"""
import numpy as np


def pooled(values, ses=None):
    v = np.asarray(values, dtype=np.float64)
    R = v.size
    se_rep = v.std(ddof=1) / np.sqrt(R) if R > 1 else 0.0
    se_delta = 0.0 if ses is None else float(np.sqrt(np.sum(np.asarray(ses, dtype=np.float64) ** 2)) / R)
    return float(v.mean()), max(se_rep, se_delta)
