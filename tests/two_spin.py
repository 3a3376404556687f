"""Exact Boltzmann averages of the two-spin open chain (N = 2, one bond) in a field.

H = -J S1.S2 - h (S1z + S2z) for unit vectors S1, S2 (Eq. 1 with a Zeeman term,
two sites).  Per site: e = H/2, m = (S1 + S2)/2, so |m|^2 = (1 + x)/2 with
x = S1.S2, and m_z = (S1z + S2z)/2.

In the polar angles theta1, theta2 and the azimuth difference psi = phi1 - phi2
the weight exp(-beta H) does not depend on phi1 + phi2, so every average is a
3-D integral: Gauss-Legendre in each theta (sin theta Jacobian included) and the
trapezoid rule in the periodic psi.  This is a test-side reference, independent
of the oracle: it samples nothing and shares no code with it.

The derivative checks need no accuracy from the quadrature itself: for any
fixed set of nodes the averages are ratios of sums of exp(-beta E_i), whose
beta and h derivatives obey the fluctuation identities exactly, so central
differences of these averages test an estimator's signs, powers of beta and
moments to the finite-difference error alone.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erfi

_NODES: dict[tuple[int, int], tuple] = {}


def _grid(n_theta: int, n_psi: int):
    key = (n_theta, n_psi)
    if key not in _NODES:
        t, w = np.polynomial.legendre.leggauss(n_theta)
        th = 0.5 * np.pi * (t + 1.0)
        wt = 0.5 * np.pi * w * np.sin(th)
        psi = 2.0 * np.pi * np.arange(n_psi) / n_psi
        u1, u2, ps = np.meshgrid(np.cos(th), np.cos(th), psi, indexing="ij")
        s1, s2, _ = np.meshgrid(np.sin(th), np.sin(th), psi, indexing="ij")
        w1, w2, _ = np.meshgrid(wt, wt, psi, indexing="ij")
        x = np.clip(u1 * u2 + s1 * s2 * np.cos(ps), -1.0, 1.0)
        _NODES[key] = (x, 0.5 * (u1 + u2), w1 * w2)
    return _NODES[key]


def moments(beta: float, J: float, h: float, n_theta: int = 96, n_psi: int = 96) -> dict[str, float]:
    """<A> for the per-site observables the records hold (mean fields only)."""
    x, mz, w = _grid(n_theta, n_psi)
    E = -J * x - 2.0 * h * mz
    a = -beta * E
    wt = w * np.exp(a - a.max())
    Z = wt.sum()
    e = 0.5 * E
    m2 = 0.5 * (1.0 + x)
    m = np.sqrt(m2)

    def avg(v):
        return float((wt * v).sum() / Z)

    return dict(e=avg(e), e2=avg(e * e), m=avg(m), m2=avg(m2), m4=avg(m2 * m2), mx=0.0, my=0.0,
                mz=avg(mz), mz2=avg(mz * mz), amz=avg(np.abs(mz)), em=avg(e * m), emz=avg(e * mz),
                mmz=avg(m * mz))


def record_rows(mom: dict[str, float], rec_fields: dict[str, int], nrec: int, rows: int = 2) -> np.ndarray:
    """Per-path records whose path means are exactly the given averages."""
    r = np.zeros((rows, nrec))
    for k, v in mom.items():
        r[:, rec_fields[k]] = v
    return r


def langevin(K: float) -> float:
    return 1.0 / np.tanh(K) - 1.0 / K


def abs_m_h0(K: float) -> float:
    """<|m|> at h = 0, K = beta J > 0, in closed form.

    x = S1.S2 has density K e^{Kx} / (2 sinh K) on [-1, 1] and
    |m| = sqrt((1 + x)/2); with y = (1 + x)/2,
    int_0^1 sqrt(y) e^{2Ky} dy = e^{2K}/(2K) - sqrt(pi) erfi(sqrt(2K)) / (2 (2K)^{3/2}).
    """
    a = 2.0 * K
    integral = np.exp(a) / a - np.sqrt(np.pi) * erfi(np.sqrt(a)) / (2.0 * a ** 1.5)
    return float(2.0 * np.exp(-K) * integral * K / (2.0 * np.sinh(K)))


def chi_h0(beta: float, J: float) -> float:
    """Eq. (cv)'s chi = (N/T)(<|m|^2> - <|m|>^2) at N = 2, h = 0, in closed form.

    J = 0: x is uniform, <|m|^2> = 1/2 and <|m|> = 2/3, so chi = beta/9.
    """
    if J == 0.0:
        return beta / 9.0
    K = beta * J
    return 2.0 * beta * (0.5 * (1.0 + langevin(K)) - abs_m_h0(K) ** 2)
