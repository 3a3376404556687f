"""Ensemble estimates from per-path records, plain numpy (test infrastructure).

Follows the paper's definitions:
  - MC average over paths, Eq. (MCAV) and Eq. (M_and_H) (Sec. 2.2);
  - <M^k> = <|M|^k>, k = 1, 2, 4 (Sec. 2.2);
  - chi = (N/T)(<|M|^2> - <|M|>^2), C_V = (N/T^2)(<H^2> - <H>^2), Eq. (cv);
  - Binder cumulant U_L = 1 - <M^4>/(3 <M^2>^2), Eq. (kum);
  - distribution coefficient r = 1 - ||R||^2 / ((n-1) sigma^2) of the normal
    Q-Q line fit, Eq. (dist-coefficient) (Sec. 3);
  - coefficient of variation of a mean cv = sigma / (sqrt(n) mean), Eq. (eq:cv).

Readings (each listed in the design notes): a path's output is the mean over
its measurement sweeps, so second moments are pooled means of per-path means
of instantaneous squares; standard errors of derived quantities are
delete-one jackknife over paths; the beta and h derivatives are the
fluctuation formulas -N cov(O, e) and beta N cov(O, m_z), plus -<m_z> in
d<e>/dh from the field term of e itself.
"""
from __future__ import annotations

import numpy as np
from scipy.special import ndtri

from .oracle import REC


def distribution_coefficient(x: np.ndarray) -> float:
    """Eq. (dist-coefficient): fit sorted data to normal quantiles by least squares.

    Plotting positions (i - 1/2)/n (the paper does not state them).
    """
    x = np.sort(np.asarray(x, dtype=np.float64))
    n = x.size
    if n < 3:
        return float("nan")
    q = ndtri((np.arange(1, n + 1) - 0.5) / n)
    A = np.vstack([np.ones(n), q]).T
    coef, *_ = np.linalg.lstsq(A, x, rcond=None)
    resid = x - A @ coef
    sigma2 = np.var(x, ddof=1)
    if sigma2 == 0.0:
        return float("nan")
    return float(1.0 - np.sum(resid ** 2) / ((n - 1) * sigma2))


def _jackknife(stat, cols: dict[str, np.ndarray]) -> float:
    """Delete-one jackknife standard error of stat(means) over paths."""
    n = next(iter(cols.values())).size
    if n < 2:
        return float("nan")
    sums = {k: v.sum() for k, v in cols.items()}
    loo = {k: (sums[k] - v) / (n - 1) for k, v in cols.items()}
    th = stat(loo)
    return float(np.sqrt((n - 1) / n * np.sum((th - th.mean()) ** 2)))


# Derived quantities of Sec. 2.2 from pooled means m (record field -> mean over
# paths), the sites per lattice N and beta = 1/T.  A Boltzmann average <A>
# under the weight exp(-beta H), H = N e, moves with the parameters as
#   d<A>/dbeta = <dA/dbeta> - cov(A, H) = -N cov(A, e)    (no A depends on beta),
#   d<A>/dh    = <dA/dh> - beta cov(A, dH/dh) = <dA/dh> + beta N cov(A, m_z),
# since dH/dh = -N m_z.  Of the observables only e = H/N depends on h itself
# (de/dh = -m_z, its Zeeman part), so d<e>/dh carries the extra -<m_z>.
def chi(m, N, beta):
    """Eq. (cv), left: (N/T) (<|m|^2> - <|m|>^2)."""
    return N * beta * (m["m2"] - m["m"] ** 2)


def cv(m, N, beta):
    """Eq. (cv), right: (N/T^2) (<e^2> - <e>^2)."""
    return N * beta ** 2 * (m["e2"] - m["e"] ** 2)


def binder(m, N, beta):
    """Eq. (kum): 1 - <|m|^4> / (3 <|m|^2>^2)."""
    return 1.0 - m["m4"] / (3.0 * m["m2"] ** 2)


def de_dbeta(m, N, beta):
    return -N * (m["e2"] - m["e"] ** 2)


def dm_dbeta(m, N, beta):
    return -N * (m["em"] - m["m"] * m["e"])


def dmz_dbeta(m, N, beta):
    return -N * (m["emz"] - m["mz"] * m["e"])


def de_dh(m, N, beta):
    return beta * N * (m["emz"] - m["e"] * m["mz"]) - m["mz"]


def dm_dh(m, N, beta):
    return beta * N * (m["mmz"] - m["m"] * m["mz"])


def dmz_dh(m, N, beta):
    return beta * N * (m["mz2"] - m["mz"] ** 2)


DERIVED = dict(chi=chi, cv=cv, binder=binder, de_dbeta=de_dbeta, dm_dbeta=dm_dbeta,
               dmz_dbeta=dmz_dbeta, de_dh=de_dh, dm_dh=dm_dh, dmz_dh=dmz_dh)


def estimates(rec: np.ndarray, N: int, T: float) -> dict[str, float]:
    """Ensemble estimates of one system from its per-path records (paths x NREC)."""
    rec = np.asarray(rec, dtype=np.float64)
    P = rec.shape[0]
    beta = 1.0 / T
    c = {k: rec[:, i] for k, i in REC.items()}
    mean = {k: float(v.mean()) for k, v in c.items()}
    se = {k: float(v.std(ddof=1) / np.sqrt(P)) if P > 1 else float("nan") for k, v in c.items()}
    out: dict[str, float] = {"n_paths": P}
    for k in ("e", "e2", "m", "m2", "m4", "mx", "my", "mz", "mz2", "amz", "acc"):
        out[k] = mean[k]
        out[k + "_se"] = se[k]

    for name, f in DERIVED.items():
        out[name] = float(f(mean, N, beta))
        out[name + "_se"] = _jackknife(lambda m, f=f: f(m, N, beta), c)

    # Eq. (eq:cv) for the order parameter <|M|>
    out["cv_m"] = se["m"] / mean["m"] if mean["m"] != 0 else float("nan")
    # Eq. (dist-coefficient) on the per-path outputs
    for k in ("e", "m", "mx", "my", "mz", "amz"):
        out["r_" + k] = distribution_coefficient(c[k])
    # Sec. 4's convergence check: the first ceil(P/2) paths and the other
    # floor(P/2) averaged separately (with the two-start scheme they started
    # from the random and from the ordered state); z = the larger of the two
    # differences (e and |m|) in units of their combined standard error.
    a = P - P // 2
    z = []
    for k in ("e", "m"):
        for half, rows in (("a", c[k][:a]), ("b", c[k][a:])):
            out[f"{k}_{half}"] = float(rows.mean()) if rows.size else float("nan")
            out[f"{k}_{half}_se"] = (float(rows.std(ddof=1) / np.sqrt(rows.size)) if rows.size > 1
                                     else float("nan"))
        d = out[f"{k}_a"] - out[f"{k}_b"]
        with np.errstate(divide="ignore", invalid="ignore"):
            z.append(np.float64(abs(d)) / np.sqrt(out[f"{k}_a_se"] ** 2 + out[f"{k}_b_se"] ** 2))
    z = [v for v in z if not np.isnan(v)]  # an undefined ratio (0/0) is skipped
    out["start_z"] = float(max(z)) if z else float("nan")
    return out
