"""The paper's literal sweep order on the GPU (Sec. 2.2: N attempts at sites
drawn at random; MP_FLAG_RANDOM_SITE) against the oracle's random-site mode,
path by path in FP64, and against the checkerboard order in distribution."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1305_6758_gb300 as mp  # noqa: E402

FIELDS = list(range(17))


def osys(s):
    return O.System(L=s.L, T=s.T, J=s.J, h=s.h, n_paths=s.n_paths, lattice=s.lattice)


def run(systems, n_therm, n_meas, seed=1, **kw):
    with mp.Simulation(systems, n_therm, n_meas, seed=seed, **kw) as sim:
        sim.run()
        recs = [sim.paths(k) for k in range(len(systems))]
        ests = [sim.estimates(k) for k in range(len(systems))]
        spins = None
        if kw.get("keep_spins"):
            spins = [np.stack([sim.spins(k, p) for p in range(s.n_paths)]) for k, s in enumerate(systems)]
    return recs, ests, spins


def test_random_site_fp64_matches_oracle():
    systems = [mp.System(4, 1.5, n_paths=64), mp.System(16, 0.7, J=-1.0, n_paths=5, lattice=mp.CHAIN),
               mp.System(6, 1.1, h=0.1, n_paths=9), mp.System(2, 0.9, n_paths=3)]
    recs, ests, spins = run(systems, 3, 4, seed=17, precision=mp.FP64, flags=mp.FLAG_RANDOM_SITE,
                            keep_spins=True)
    refs, rsp = O.run([osys(s) for s in systems], 3, 4, seed=17, order_mode=O.ORDER_RANDOM, want_spins=True)
    for s, g, r, gs, os_, e in zip(systems, recs, refs, spins, rsp, ests):
        np.testing.assert_array_equal(g[:, 17], r[:, 17])
        assert np.abs(gs - os_).max() < 1e-12
        np.testing.assert_allclose(g[:, FIELDS], r[:, FIELDS], rtol=1e-10, atol=1e-13)
        o = O.estimates(r, s.N, s.T)
        for k in ("e", "m", "chi", "cv"):
            assert e[k] == pytest.approx(o[k], rel=1e-8, abs=1e-12), k


def test_random_site_plain_config_matches_checkerboard():
    """The plain-method configuration (L = 4, T = 1.5, 256 paths, 1000 + 1000
    sweeps) in both orders: ensemble means agree within 4 combined SE."""
    s = [mp.System(4, 1.5, n_paths=256)]
    _, a, _ = run(s, 1000, 1000, seed=3, flags=mp.FLAG_RANDOM_SITE)
    _, b, _ = run(s, 1000, 1000, seed=4)
    for k in ("e", "m", "m2"):
        assert abs(a[0][k] - b[0][k]) < 4 * np.hypot(a[0][k + "_se"], b[0][k + "_se"]), k


def test_random_site_rejections():
    with mp.Simulation([mp.System(4, 1.5, n_paths=4)], 1, 1, flags=mp.FLAG_RANDOM_SITE) as sim:
        with pytest.raises(mp.MPError) as ei:
            sim.run_sweeps(1)
        assert ei.value.status == mp.MP_EINVAL
    with pytest.raises(mp.MPError) as ei:
        mp.Simulation([mp.System(4, 1.5, n_paths=4, lattice=mp.ISING)], 1, 1, flags=mp.FLAG_RANDOM_SITE)
    assert ei.value.status == mp.MP_EINVAL
