"""Pins of the oracle's 2D Ising path (Appendix A), each against something
other than the oracle itself: exact enumeration of the 4 x 4 periodic
lattice, Onsager's energy and Yang's spontaneous magnetisation of the
infinite lattice, independent spins in a field, and the T -> 0 and T -> inf
limits.
"""
import numpy as np
import pytest
from scipy.special import ellipk

import oracle as O


def zdiff(a, b, se):
    return abs(a - b) / se


def enumerate_4x4(T, J=1.0, h=0.0):
    """Exact Boltzmann averages over all 2^16 states of the periodic 4 x 4 lattice."""
    L, N = 4, 16
    idx = np.arange(2 ** N, dtype=np.int64)
    s = 1 - 2 * ((idx[:, None] >> np.arange(N)) & 1)  # (states, sites), +-1
    s = s.reshape(-1, L, L)  # [state, y, x]
    bonds = (s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) + (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    M = s.sum(axis=(1, 2))
    E = -J * bonds - h * M
    w = np.exp(-(E - E.min()) / T)
    w /= w.sum()
    e, m = E / N, M / N
    avg = lambda x: float((w * x).sum())  # noqa: E731
    out = dict(e=avg(e), e2=avg(e * e), m=avg(np.abs(m)), m2=avg(m * m), m4=avg(m ** 4), mz=avg(m))
    out["chi"] = N / T * (out["m2"] - out["m"] ** 2)
    out["cv"] = N / T ** 2 * (out["e2"] - out["e"] ** 2)
    out["binder"] = 1 - out["m4"] / (3 * out["m2"] ** 2)
    return out


@pytest.mark.parametrize("T,h", [(2.5, 0.0), (2.0, 0.2), (3.5, -0.3)])
def test_ising_4x4_exact_enumeration(T, h):
    rec = O.run([O.System(L=4, T=T, h=h, n_paths=4096, lattice=O.ISING)], 300, 300, seed=7)[0]
    est = O.estimates(rec, 16, T)
    ex = enumerate_4x4(T, h=h)
    for k in ("e", "e2", "m", "m2", "m4", "mz", "chi", "cv", "binder"):
        assert zdiff(est[k], ex[k], est[k + "_se"]) < 4.5, (k, est[k], ex[k], est[k + "_se"])


def onsager_energy(T, J=1.0):
    """Energy per site of the infinite square-lattice Ising model (Onsager)."""
    K = J / T
    k = 2 * np.sinh(2 * K) / np.cosh(2 * K) ** 2
    return -J / np.tanh(2 * K) * (1 + 2 / np.pi * (2 * np.tanh(2 * K) ** 2 - 1) * ellipk(k * k))


def yang_magnetisation(T, J=1.0):
    return (1 - np.sinh(2 * J / T) ** -4) ** 0.125


def test_ising_onsager_yang_large_lattice():
    """L = 32 away from T_C = 2.269: finite-size corrections are exponentially small."""
    lo = O.estimates(O.run([O.System(L=32, T=2.0, n_paths=32, lattice=O.ISING)], 500, 1000, seed=3,
                           init_mode=O.INIT_ORDERED)[0], 1024, 2.0)
    hi = O.estimates(O.run([O.System(L=32, T=3.0, n_paths=32, lattice=O.ISING)], 500, 1000, seed=4)[0],
                     1024, 3.0)
    assert abs(lo["e"] - onsager_energy(2.0)) < 4 * lo["e_se"] + 1e-3
    assert abs(lo["m"] - yang_magnetisation(2.0)) < 4 * lo["m_se"] + 1e-3
    assert abs(hi["e"] - onsager_energy(3.0)) < 4 * hi["e_se"] + 1e-3
    assert hi["m"] < 0.1  # paramagnet: <|m|> ~ N^-1/2


def test_ising_free_spins_in_field():
    """J = 0: independent spins, <s> = tanh(beta h), Var(m) = (1 - tanh^2) / N."""
    T, h, N = 1.0, 0.3, 16
    est = O.estimates(O.run([O.System(L=4, T=T, J=0.0, h=h, n_paths=2048, lattice=O.ISING)], 20, 200)[0],
                      N, T)
    t = np.tanh(h / T)
    assert zdiff(est["mz"], t, est["mz_se"]) < 4
    assert zdiff(est["mz2"], t * t + (1 - t * t) / N, est["mz2_se"]) < 4
    assert est["e"] == pytest.approx(-h * est["mz"], rel=1e-12)


def test_ising_limits():
    cold = O.run([O.System(L=6, T=1e-300, n_paths=3, lattice=O.ISING)], 0, 4, init_mode=O.INIT_ORDERED)[0]
    assert np.all(cold[:, O.REC["e"]] == -2.0) and np.all(cold[:, O.REC["acc"]] == 0.0)
    assert np.all(cold[:, O.REC["m"]] == 1.0)
    hot = O.run([O.System(L=6, T=1e300, n_paths=3, lattice=O.ISING)], 2, 2)[0]
    assert np.all(hot[:, O.REC["acc"]] == 1.0)
    # every flip accepted: after an even number of sweeps the random start returns
    _, sp = O.run([O.System(L=6, T=1e300, n_paths=2, lattice=O.ISING)], 0, 2, want_spins=True)
    _, sp0 = O.run([O.System(L=6, T=1e300, n_paths=2, lattice=O.ISING)], 0, 1, want_spins=True)
    assert np.all(np.abs(sp[0][:, :, 2]) == 1.0)
    assert np.all(sp0[0][:, :, 2] == -sp[0][:, :, 2])


def test_ising_two_start_and_odd_size_rejected():
    rec = O.run([O.System(L=8, T=1.5, n_paths=10, lattice=O.ISING)], 0, 1, two_start=True)[0]
    assert np.all(rec[5:, O.REC["fmz"]] > 0.9)  # ordered half, one sweep at T = 1.5
    with pytest.raises(ValueError):
        O.run([O.System(L=5, T=1.5, n_paths=1, lattice=O.ISING)], 1, 1)
