"""The FP32 simple cubic L = 32 lattice held by the two CTAs of a cluster.

Each CTA keeps half of the z-planes in shared memory plus one halo plane per
colour on either side, filled by the partner through distributed shared
memory; one cluster barrier per half-sweep.  The per-site arithmetic is that
of every other FP32 kernel and the neighbour sums keep the fixed order, so a
path follows the trajectory of the same path streamed from HBM (to FP32
rounding of the partial sums) and, after a few sweeps, the FP64 oracle's.
"""
import time

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1305_6758_gb300 as mp  # noqa: E402

FIELDS = list(range(17))


def osys(s, **kw):
    return O.System(L=s.L, T=s.T, J=s.J, h=s.h, n_paths=s.n_paths, lattice=s.lattice, **kw)


def test_l32_fp32_runs_on_two_cta_clusters():
    with mp.Simulation([mp.System(32, 1.4, n_paths=3), mp.System(8, 1.0, n_paths=5)], 1, 1) as sim:
        a, b = sim.system_plan(0), sim.system_plan(1)
        plan = sim.plan()
    assert a["cluster_pair"] and not a["streamed"] and a["paths_per_cta"] == 1
    assert not b["cluster_pair"]
    assert plan["grid"] % 2 == 0
    with mp.Simulation([mp.System(32, 1.4, n_paths=3)], 1, 1, flags=mp.FLAG_STREAM) as sim:
        assert sim.system_plan(0)["streamed"]
    with mp.Simulation([mp.System(32, 1.4, n_paths=3)], 1, 1, precision=mp.FP64) as sim:
        assert not sim.system_plan(0)["cluster_pair"]


@pytest.mark.parametrize("init", [mp.INIT_SPHERE, mp.INIT_ANGLES, mp.INIT_ORDERED])
def test_cluster_follows_the_streamed_trajectory(init):
    systems = [mp.System(32, 1.3, h=0.05, n_paths=5), mp.System(32, 0.7, J=-1.0, n_paths=3)]
    kw = dict(seed=9, init_mode=init, keep_spins=True)
    with mp.Simulation(systems, 3, 4, **kw) as a, \
            mp.Simulation(systems, 3, 4, flags=mp.FLAG_STREAM, **kw) as b:
        a.run()
        b.run()
        assert a.system_plan(0)["cluster_pair"] and b.system_plan(0)["streamed"]
        for k, s in enumerate(systems):
            ra, rb = a.paths(k), b.paths(k)
            np.testing.assert_allclose(ra[:, FIELDS], rb[:, FIELDS], rtol=0, atol=2e-5)
            np.testing.assert_array_equal(ra[:, 17], rb[:, 17])  # acceptance counts
            for p in range(s.n_paths):
                np.testing.assert_allclose(a.spins(k, p), b.spins(k, p), rtol=0, atol=2e-5)


@pytest.mark.parametrize("sweeps", [(0, 1), (1, 2)])
def test_cluster_against_the_oracle(sweeps):
    """Path by path against the FP64 oracle: FP32 rounding may flip a
    borderline acceptance in at most one of the paths."""
    systems = [mp.System(32, 1.44, n_paths=4)]
    with mp.Simulation(systems, *sweeps, seed=3) as sim:
        sim.run()
        got = sim.paths(0)
    ref = O.run([osys(systems[0])], *sweeps, seed=3)[0]
    bad = sum(int(np.max(np.abs(g[FIELDS] - r[FIELDS])) > 1e-5) for g, r in zip(got, ref))
    assert bad <= 1, f"{bad} of 4 paths differ"


def test_cluster_paths_in_an_uneven_batch():
    """In a batch with single-CTA sizes the mixed-size kernel runs the L = 32
    paths first on clusters, then the rest: the same records as L = 32 alone."""
    alone = [mp.System(32, 1.2, n_paths=6)]
    batch = [mp.System(8, 1.0, n_paths=300), mp.System(32, 1.2, n_paths=6), mp.System(16, 0.9, n_paths=40)]
    with mp.Simulation(alone, 2, 3, seed=12) as a:
        a.run()
        ra = a.paths(0)
    with mp.Simulation(batch, 2, 3, seed=12) as b:
        b.run()
        rb = b.paths(1)
        assert b.system_plan(1)["cluster_pair"]
    # system index 1 in the batch: other random numbers than system 0 alone
    with mp.Simulation([mp.System(8, 1.0, n_paths=1), alone[0]], 2, 3, seed=12) as c:
        c.run()
        rc = c.paths(1)
    np.testing.assert_allclose(rb[:, FIELDS], rc[:, FIELDS], rtol=0, atol=2e-6)
    assert not np.allclose(ra[:, 0], rb[:, 0])


def test_cluster_split_schedule_with_checkpoint_equals_one_run():
    systems = [mp.System(32, 1.4, n_paths=5), mp.System(8, 1.1, n_paths=20)]
    with mp.Simulation(systems, 4, 5, seed=6) as whole:
        whole.run_sweeps(9)
        ref = [whole.paths(k) for k in range(2)]
    with mp.Simulation(systems, 4, 5, seed=6) as a:
        a.run_sweeps(3)
        a.run_sweeps(3)
        blob = a.checkpoint()
    with mp.Simulation(systems, 4, 5, seed=6) as b:
        b.restore(blob)
        b.run_sweeps(100)
        got = [b.paths(k) for k in range(2)]
    for r, g in zip(ref, got):
        np.testing.assert_allclose(g[:, FIELDS], r[:, FIELDS], rtol=0, atol=1e-6)
        np.testing.assert_array_equal(g[:, 17], r[:, 17])


def test_cluster_two_start_halves():
    """Sec. 4's two starts: the first ceil(P/2) paths equal the single-start
    run, the others the ordered-start run."""
    s = [mp.System(32, 1.0, n_paths=5)]
    recs = {}
    for name, kw in (("two", dict(flags=mp.FLAG_TWO_START)), ("rnd", {}), ("ord", dict(init_mode=mp.INIT_ORDERED))):
        with mp.Simulation(s, 1, 2, seed=4, **kw) as sim:
            sim.run()
            recs[name] = sim.paths(0)
    np.testing.assert_allclose(recs["two"][:3, FIELDS], recs["rnd"][:3, FIELDS], rtol=0, atol=1e-6)
    np.testing.assert_allclose(recs["two"][3:, FIELDS], recs["ord"][3:, FIELDS], rtol=0, atol=1e-6)


def test_cluster_cancel_stops_both_ctas():
    sim = mp.Simulation([mp.System(32, 1.0, n_paths=2048)], 3000, 3000, graph=False)  # ~60 s if not stopped
    t0 = time.time()
    sim.run()
    time.sleep(0.2)
    sim.cancel()
    with pytest.raises(mp.MPError) as ei:
        sim.estimates(0)
    assert ei.value.status == mp.MP_ECANCELED
    assert time.time() - t0 < 10.0
    sim.close()
    with mp.Simulation([mp.System(32, 1.5, n_paths=4)], 2, 2) as ok:
        ok.run()
        assert np.isfinite(ok.estimates(0)["e"])


def test_every_lattice_mode_in_one_launch():
    """One FP32 batch with a lattice of each mode (two-CTA cluster L = 32,
    streamed L = 64, in place L = 66, shared memory L = 8): the mixed-size
    kernel, launched in clusters, dispatches each; every path against the
    oracle after two sweeps (a borderline acceptance may flip one path)."""
    systems = [mp.System(32, 1.4, n_paths=3), mp.System(64, 1.44, n_paths=2), mp.System(66, 1.5, n_paths=2),
               mp.System(8, 1.0, n_paths=5)]
    with mp.Simulation(systems, 1, 1, seed=14) as sim:
        sim.run()
        plans = [sim.system_plan(k) for k in range(len(systems))]
        got = [sim.paths(k) for k in range(len(systems))]
    assert plans[0]["cluster_pair"] and plans[1]["streamed"] and plans[2]["in_place_hbm"]
    assert not (plans[3]["cluster_pair"] or plans[3]["streamed"] or plans[3]["in_place_hbm"])
    refs = O.run([osys(s) for s in systems], 1, 1, seed=14)
    for s, g, r in zip(systems, got, refs):
        bad = sum(int(np.max(np.abs(a[FIELDS] - b[FIELDS])) > 1e-5) for a, b in zip(g, r))
        assert bad <= 1, (s.L, bad)
