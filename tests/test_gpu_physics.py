"""Physics checks of the paper on the GPU path (FP32 form, paper-sized runs).

Sec. 4: half the paths from the random state and half from the ordered state
converge to the same estimates (the two-start check), and so do the three
initial states (uniform on the sphere, uniform angles, ordered).  Sec. 5: the
Binder cumulants of L = 20 and L = 30 cross near T_C = 1.442(20).  The FP64
form of the two-start scheme is compared with the oracle path by path.
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
        return [sim.paths(k) for k in range(len(systems))], [sim.estimates(k) for k in range(len(systems))]


def test_two_start_fp64_matches_oracle():
    systems = [mp.System(6, 1.0, n_paths=9), mp.System(16, 0.8, n_paths=6, lattice=mp.CHAIN),
               mp.System(24, 1.2, n_paths=3)]  # the last one streamed
    recs, ests = run(systems, 2, 3, seed=6, precision=mp.FP64, flags=mp.FLAG_TWO_START)
    refs = O.run([O.System(L=s.L, T=s.T, n_paths=s.n_paths, lattice=s.lattice) for s in systems], 2, 3,
                 seed=6, two_start=True)
    for s, g, r, e in zip(systems, recs, refs, ests):
        np.testing.assert_allclose(g[:, FIELDS], r[:, FIELDS], rtol=1e-10, atol=1e-13)
        o = O.estimates(r, s.L ** 3 if s.lattice == mp.SC else s.L, s.T)
        for k in ("e_a", "e_a_se", "e_b", "e_b_se", "m_a", "m_a_se", "m_b", "m_b_se", "start_z"):
            assert e[k] == pytest.approx(o[k], rel=1e-8, abs=1e-12, nan_ok=True), k


def test_two_start_check_l10_t1():
    """L = 10, T = 1 (ordered phase): random and ordered halves differ after one
    sweep and agree after thermalisation."""
    s = [mp.System(10, 1.0, n_paths=4096)]
    _, early = run(s, 0, 1, flags=mp.FLAG_TWO_START)
    assert early[0]["start_z"] > 20 and early[0]["e_b"] < early[0]["e_a"]
    _, late = run(s, 2000, 1000, flags=mp.FLAG_TWO_START)
    assert late[0]["start_z"] < 4, late[0]


def test_three_initial_states_converge():
    s = [mp.System(10, 1.0, n_paths=2048)]
    res = {m: run(s, 2000, 1000, seed=3 + m, init_mode=m)[1][0]
           for m in (mp.INIT_SPHERE, mp.INIT_ANGLES, mp.INIT_ORDERED)}
    for a in res.values():
        for b in res.values():
            for k in ("e", "m"):
                assert abs(a[k] - b[k]) < 4 * np.hypot(a[k + "_se"], b[k + "_se"]) + 1e-12


def test_table1_distribution_coefficients_l10():
    """Sec. 3, Table 1: L = 10, 10^4 paths, each path's output its final state
    (n_meas = 1, as in the paper).  The energy is normal at every temperature
    of the table (r at least the printed value less 0.005), and so are the
    spin components in the disordered phase (T = 1.6).  In the ordered phase
    the trial move uniform on the sphere leaves the direction of the total
    spin isotropic, so each component is |M| times a uniform cosine and r
    is that of a uniform sample, 3/pi; the table's 0.9998 there reflects a
    parametrisation that favours the poles, which is not reproduced."""
    table = golden.table1()
    Ts = sorted(table)
    systems = [mp.System(10, T, n_paths=10000) for T in Ts]
    _, ests = run(systems, 3000, 1, seed=12)
    for T, e in zip(Ts, ests):
        print(T, {k: (round(e[k], 4), ref) for k, ref in table[T].items()})
    for T, e in zip(Ts, ests):
        assert e["r_e"] > table[T]["r_e"] - 0.005, (T, e["r_e"])
        if T <= 1.0:
            for k in ("r_mx", "r_my"):
                assert abs(e[k] - 3 / np.pi) < 0.01, (T, k, e[k])
        if T >= 1.6:
            for k in ("r_mx", "r_my", "r_mz"):
                assert e[k] > table[T][k] - 0.005, (T, k, e[k])


def test_binder_cumulant_crossing():
    """U_L for L = 20 and L = 30 in one batched launch (L = 30 streamed): the
    curves cross inside the paper's T_C = 1.442 +- 0.020 (Sec. 5)."""
    l_small, l_large, tc_paper, tc_err = golden.critical_temperature("heisenberg_sc")
    Ts = [1.40, 1.42, 1.44, 1.46, 1.48]
    systems = [mp.System(L, T, n_paths=4096) for L in (l_small, l_large) for T in Ts]
    _, ests = run(systems, 1000, 1000, seed=21)
    u20 = np.array([e["binder"] for e in ests[:5]])
    u30 = np.array([e["binder"] for e in ests[5:]])
    se = np.hypot([e["binder_se"] for e in ests[:5]], [e["binder_se"] for e in ests[5:]])
    d = u30 - u20
    print("U20", u20, "U30", u30, "d/se", d / se)
    assert d[0] > 3 * se[0] and d[-1] < -3 * se[-1]
    k = int(np.nonzero((d[:-1] > 0) & (d[1:] <= 0))[0][0])
    tc = Ts[k] + (Ts[k + 1] - Ts[k]) * d[k] / (d[k] - d[k + 1])
    print("crossing", tc)
    assert abs(tc - tc_paper) < tc_err
