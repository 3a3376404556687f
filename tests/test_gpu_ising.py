"""GPU parity of the square-lattice Ising path (Appendix A) against the oracle.

The device test is an integer compare against thresholds computed in FP64
from the same definition, so final spins and acceptance counts are
bit-identical to the oracle; per-path FP64 means agree to rounding.  Then
the appendix's physics at paper-like sizes: Onsager-Yang below T_C, and the
Binder cumulants of L = 50 and 60 crossing near T_C = 2.269.
"""
import numpy as np
import pytest

import golden
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1305_6758_gb300 as mp  # noqa: E402

FIELDS = list(range(17))


def run(systems, n_therm, n_meas, seed=1, **kw):
    with mp.Simulation(systems, n_therm, n_meas, seed=seed, **kw) as sim:
        sim.run()
        recs = [sim.paths(k) for k in range(len(systems))]
        ests = [sim.estimates(k) for k in range(len(systems))]
        spins = None
        if kw.get("keep_spins"):
            spins = [np.stack([sim.spins(k, p) for p in range(s.n_paths)]) for k, s in enumerate(systems)]
    return recs, ests, spins


def osys(s):
    return O.System(L=s.L, T=s.T, J=s.J, h=s.h, n_paths=s.n_paths, lattice=O.ISING)


@pytest.mark.parametrize("systems,init,two", [
    ([mp.System(8, 2.3, n_paths=37, lattice=mp.ISING)], mp.INIT_SPHERE, False),
    ([mp.System(2, 1.0, h=0.4, n_paths=5, lattice=mp.ISING), mp.System(10, 1.7, J=-1.0, n_paths=9, lattice=mp.ISING),
      mp.System(50, 2.269, h=-0.05, n_paths=4, lattice=mp.ISING)], mp.INIT_SPHERE, False),
    ([mp.System(20, 1.5, n_paths=6, lattice=mp.ISING)], mp.INIT_ORDERED, False),
    ([mp.System(6, 2.0, n_paths=7, lattice=mp.ISING)], mp.INIT_SPHERE, True),
])
def test_ising_matches_oracle_exactly(systems, init, two):
    flags = mp.FLAG_TWO_START if two else 0
    recs, ests, spins = run(systems, 5, 7, seed=13, init_mode=init, flags=flags, keep_spins=True)
    refs, rsp = O.run([osys(s) for s in systems], 5, 7, seed=13, init_mode=init, two_start=two,
                      want_spins=True)
    for s, g, r, gs, os_, e in zip(systems, recs, refs, spins, rsp, ests):
        np.testing.assert_array_equal(gs, os_)            # final spins, bit for bit
        np.testing.assert_array_equal(g[:, 17], r[:, 17])  # acceptance counts
        np.testing.assert_allclose(g[:, FIELDS], r[:, FIELDS], rtol=1e-12, atol=1e-14)
        o = O.estimates(r, s.L * s.L, s.T)
        for k in ("e", "m", "chi", "cv", "binder", "start_z"):
            assert e[k] == pytest.approx(o[k], rel=1e-9, abs=1e-12, nan_ok=True), k


def test_ising_full_size_first_sweeps_and_layouts():
    """A paper-sized launch (L = 60, 10^4 paths) for two sweeps: sampled paths
    equal the oracle bit for bit; a forced thread layout changes nothing."""
    s = [mp.System(60, 2.269, n_paths=10000, lattice=mp.ISING)]
    recs, _, _ = run(s, 1, 1, seed=2)
    idx = [0, 1, 4999, 9998, 9999]
    for p in idx:
        ref = O.run([O.System(L=60, T=2.269, n_paths=10000, path_begin=p, path_count=1, lattice=O.ISING)],
                    1, 1, seed=2)[0][0]
        np.testing.assert_allclose(recs[0][p, FIELDS], ref[FIELDS], rtol=1e-12, atol=1e-14)
        assert recs[0][p, 17] == ref[17]
    for tp in (32, 96, 256):
        r2, _, _ = run(s, 1, 1, seed=2, threads_per_path=tp)
        np.testing.assert_array_equal(r2[0], recs[0])


def onsager_energy(T):
    from scipy.special import ellipk
    K = 1.0 / T
    k = 2 * np.sinh(2 * K) / np.cosh(2 * K) ** 2
    return -1 / np.tanh(2 * K) * (1 + 2 / np.pi * (2 * np.tanh(2 * K) ** 2 - 1) * ellipk(k * k))


def test_ising_onsager_yang_paper_sizes():
    """Appendix A, Fig. a: <|m|> below T_C on L = 40 and 60 against Yang's
    spontaneous magnetisation, <e> against Onsager (ordered start)."""
    Ts = (1.5, 1.8, 2.0)
    systems = [mp.System(L, T, n_paths=1024, lattice=mp.ISING) for L in (40, 60) for T in Ts]
    _, ests, _ = run(systems, 1000, 1000, seed=5, init_mode=mp.INIT_ORDERED)
    for s, e in zip(systems, ests):
        yang = (1 - np.sinh(2 / s.T) ** -4) ** 0.125
        assert abs(e["m"] - yang) < 4 * e["m_se"] + 2e-3, (s.L, s.T, e["m"], yang)
        assert abs(e["e"] - onsager_energy(s.T)) < 4 * e["e_se"] + 2e-3, (s.L, s.T, e["e"])


def test_ising_binder_crossing():
    """Appendix A: U_L of L = 50 and 60 cross inside the paper's T_C = 2.269(10):
    the larger lattice's U_L is above the smaller one's by 3 standard errors
    below T_C and below it by 3 above T_C, and the interpolated crossing lies
    within the printed error."""
    l_small, l_large, tc_paper, tc_err = golden.critical_temperature("ising_square")
    Ts = [2.24, 2.26, 2.28, 2.30]
    systems = [mp.System(L, T, n_paths=8192, lattice=mp.ISING) for L in (l_small, l_large) for T in Ts]
    _, ests, _ = run(systems, 20000, 10000, seed=9)  # the appendix's 3 x 10^4 sweeps
    u50 = np.array([e["binder"] for e in ests[:4]])
    u60 = np.array([e["binder"] for e in ests[4:]])
    se = np.hypot([e["binder_se"] for e in ests[:4]], [e["binder_se"] for e in ests[4:]])
    d = u60 - u50
    print("U50", u50, "U60", u60, "d/se", d / se)
    assert d[0] > 3 * se[0] and d[-1] < -3 * se[-1]
    k = int(np.nonzero((d[:-1] > 0) & (d[1:] <= 0))[0][0])
    tc = Ts[k] + (Ts[k + 1] - Ts[k]) * d[k] / (d[k] - d[k + 1])
    print("crossing", tc)
    assert abs(tc - tc_paper) < tc_err
