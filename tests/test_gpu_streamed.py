"""The HBM-streamed sweep (lattices too large for shared memory).

Its z-plane wavefront gives every update the neighbour values of the
two-pass checkerboard sweep, so the FP64 form reproduces the oracle path by
path, and a lattice forced through the streamed kernel follows the same
trajectory as in the shared-memory kernel.
"""
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


def gpu_records(systems, n_therm, n_meas, seed=1, **kw):
    with mp.Simulation(systems, n_therm, n_meas, seed=seed, **kw) as sim:
        sim.run()
        plan = sim.plan()
        return [sim.paths(k) for k in range(len(systems))], plan


@pytest.mark.parametrize("systems", [
    [mp.System(22, 1.2, n_paths=3)],
    [mp.System(28, 0.9, h=0.05, n_paths=2)],
    [mp.System(32, 1.44, J=-1.0, n_paths=2)],
])
def test_streamed_fp64_matches_oracle(systems):
    recs, _ = gpu_records(systems, 2, 3, seed=5, precision=mp.FP64)
    refs = O.run([osys(s) for s in systems], 2, 3, seed=5)
    for g, r in zip(recs, refs):
        np.testing.assert_allclose(g[:, FIELDS], r[:, FIELDS], rtol=1e-10, atol=1e-13)
        np.testing.assert_array_equal(g[:, 17], r[:, 17])


def test_uneven_batch_shared_and_streamed_in_one_launch_fp64():
    """Batched uneven sizes (L = 8 ... 32) in one persistent launch: sizes up to 20
    in shared memory, 24 and 32 streamed; every path against the oracle."""
    systems = [mp.System(L, 1.44, n_paths=P) for L, P in ((8, 16), (12, 8), (16, 4), (20, 2), (24, 2), (32, 1))]
    recs, plan = gpu_records(systems, 2, 2, seed=3, precision=mp.FP64)
    refs = O.run([osys(s) for s in systems], 2, 2, seed=3)
    for g, r in zip(recs, refs):
        np.testing.assert_allclose(g[:, FIELDS], r[:, FIELDS], rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("sweeps", [(0, 1), (1, 1), (2, 3)])
def test_streamed_many_paths_per_cta(sweeps):
    """Each persistent CTA runs many streamed paths in turn (its mbarriers are
    re-armed per path); odd and even numbers of loads per ring slot."""
    systems = [mp.System(24, 1.1, n_paths=1200)]
    recs, plan = gpu_records(systems, *sweeps, seed=2, precision=mp.FP64, flags=mp.FLAG_STREAM)
    assert plan["n_items"] > plan["grid"], plan
    refs = O.run([osys(s) for s in systems], *sweeps, seed=2)
    np.testing.assert_allclose(recs[0][:, FIELDS], refs[0][:, FIELDS], rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("precision", [mp.FP64, mp.FP32])
def test_forced_streaming_follows_shared_memory_trajectory(precision):
    systems = [mp.System(16, 1.3, n_paths=6), mp.System(8, 0.8, h=0.02, n_paths=10), mp.System(4, 2.0, n_paths=9)]
    with mp.Simulation(systems, 3, 4, seed=8, precision=precision, keep_spins=True) as a, \
            mp.Simulation(systems, 3, 4, seed=8, precision=precision, keep_spins=True, flags=mp.FLAG_STREAM) as b:
        a.run()
        b.run()
        for k, s in enumerate(systems):
            ra, rb = a.paths(k), b.paths(k)
            tol = 1e-12 if precision == mp.FP64 else 2e-5
            np.testing.assert_allclose(ra[:, FIELDS], rb[:, FIELDS], rtol=0, atol=tol)
            for p in range(s.n_paths):
                np.testing.assert_allclose(a.spins(k, p), b.spins(k, p), rtol=0, atol=tol)


def test_full_size_l64_launch_first_sweep():
    """The large-lattice launch (L = 64, 3 temperatures x 1024 paths, FP32) after one
    sweep: sampled paths of each system against the oracle."""
    Ts = [1.40, 1.44, 1.48]
    systems = [mp.System(64, T, n_paths=1024) for T in Ts]
    recs, plan = gpu_records(systems, 0, 1, seed=1)
    bad = total = 0
    for begin in (0, 511, 1023):
        refs = O.run([O.System(64, T, n_paths=1024, path_begin=begin, path_count=1) for T in Ts], 0, 1)
        for k in range(3):
            total += 1
            bad += int(np.max(np.abs(recs[k][begin][FIELDS] - refs[k][0][FIELDS])) > 1e-5)
    assert bad <= 1, f"{bad} of {total} sampled paths differ"


@pytest.mark.parametrize("tp", [256, 384, 512])
def test_l64_kernel_every_row_layout(tp):
    """The kernel compiled for L = 64: 16 row groups (compile-time rows), 8 and
    12 row groups (rows at run time): two sweeps of a few paths against the oracle."""
    systems = [mp.System(64, 1.44, n_paths=3)]
    recs, _ = gpu_records(systems, 1, 1, seed=6, threads_per_path=tp)
    refs = O.run([osys(systems[0])], 1, 1, seed=6)
    bad = sum(int(np.max(np.abs(g[FIELDS] - r[FIELDS])) > 1e-5) for g, r in zip(recs[0], refs[0]))
    assert bad <= 1, f"{bad} of 3 paths differ"


def test_stalled_bulk_copy_reports_timeout():
    """Failure detection: a bulk copy that is never issued makes the bounded
    mbarrier wait give up (about 2 s); the host reads MP_ETIMEOUT, the context
    stays usable."""
    sim = mp.Simulation([mp.System(8, 1.0, n_paths=1)], 1, 1, flags=mp.FLAG_STREAM | mp.FLAG_TEST_STALL)
    sim.run()
    with pytest.raises(mp.MPError) as ei:
        sim.estimates(0)
    assert ei.value.status == mp.MP_ETIMEOUT
    sim.close()
    # the device still works
    with mp.Simulation([mp.System(8, 1.0, n_paths=4)], 1, 1, flags=mp.FLAG_STREAM) as ok:
        ok.run()
        assert np.isfinite(ok.estimates(0)["e"])


@pytest.mark.parametrize("systems", [
    [mp.System(64, 1.44, n_paths=2)],                                      # the in-place kernel
    [mp.System(46, 0.9, h=0.05, n_paths=2), mp.System(8, 1.0, n_paths=3)],  # with a shared-memory size
    [mp.System(46, 1.2, J=-1.0, n_paths=2), mp.System(24, 1.1, n_paths=2)],  # with a streamed size
])
def test_in_place_fp64_matches_oracle(systems):
    """FP64 lattices whose half-plane ring does not fit shared memory (L >= 46)
    are updated in place in HBM: path by path equal to the oracle."""
    with mp.Simulation(systems, 1, 2, seed=5, precision=mp.FP64) as sim:
        sim.run()
        recs = [sim.paths(k) for k in range(len(systems))]
        assert sim.system_plan(0)["in_place_hbm"]
    refs = O.run([osys(s) for s in systems], 1, 2, seed=5)
    for g, r in zip(recs, refs):
        np.testing.assert_allclose(g[:, FIELDS], r[:, FIELDS], rtol=1e-10, atol=1e-13)
        np.testing.assert_array_equal(g[:, 17], r[:, 17])


def test_in_place_fp32_l66_against_oracle():
    systems = [mp.System(66, 1.44, n_paths=2)]
    with mp.Simulation(systems, 0, 1, seed=7) as sim:
        sim.run()
        got = sim.paths(0)
        assert sim.system_plan(0)["in_place_hbm"]
    ref = O.run([osys(systems[0])], 0, 1, seed=7)[0]
    bad = sum(int(np.max(np.abs(g[FIELDS] - r[FIELDS])) > 1e-5) for g, r in zip(got, ref))
    assert bad <= 1


def test_autotune_changes_only_the_launch_shape():
    """MP_FLAG_AUTOTUNE times candidate layouts; the trajectories (and FP64
    records) do not depend on the layout it keeps."""
    systems = [mp.System(12, 1.2, n_paths=300), mp.System(8, 1.0, n_paths=500), mp.System(28, 1.4, n_paths=3)]
    a, pa = gpu_records(systems, 2, 2, seed=4, precision=mp.FP64)
    b, pb = gpu_records(systems, 2, 2, seed=4, precision=mp.FP64, flags=mp.FLAG_AUTOTUNE)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x[:, FIELDS], y[:, FIELDS], rtol=1e-12, atol=1e-14)
    with mp.Simulation(systems, 1, 1, flags=mp.FLAG_AUTOTUNE) as sim:
        shapes = [sim.system_plan(k) for k in range(3)]
    assert shapes[2]["streamed"] and not shapes[0]["streamed"]
    assert all(s["threads_per_path"] % 32 == 0 for s in shapes)


def test_autotune_choice_is_remembered_for_the_same_batch_shape():
    """A second handle of the same batch shape takes the first one's measured
    layout (no timing at create); another temperature does not change the key."""
    import time
    systems = [mp.System(10, 1.3, n_paths=700), mp.System(14, 0.9, n_paths=90)]
    t0 = time.perf_counter()
    with mp.Simulation(systems, 1, 1, flags=mp.FLAG_AUTOTUNE, seed=3) as a:
        first = [a.system_plan(k) for k in range(2)], a.plan()
    t1 = time.perf_counter()
    hot = [mp.System(10, 2.0, n_paths=700), mp.System(14, 1.1, n_paths=90)]
    with mp.Simulation(hot, 1, 1, flags=mp.FLAG_AUTOTUNE, seed=4) as b:
        again = [b.system_plan(k) for k in range(2)], b.plan()
    t2 = time.perf_counter()
    assert again == first
    assert t2 - t1 < t1 - t0


def test_fp32_batched_form_against_the_oracle():
    """The batched workload's shape in FP32: uneven sizes in one persistent
    launch, L = 32 on two-CTA clusters, autotuned. Every system's <e> and <|m|> are
    within 3 combined standard errors of the FP64 oracle, and <e> is within
    1e-4 (plus 3 standard errors) of the FP64 GPU form from the same starts."""
    sizes = ((8, 512), (12, 256), (16, 128), (20, 64), (24, 32), (32, 16))
    systems = [mp.System(L, 1.44, n_paths=P) for L, P in sizes]
    with mp.Simulation(systems, 100, 100, seed=11, flags=mp.FLAG_AUTOTUNE) as sim:
        sim.run()
        e32 = [sim.estimates(k) for k in range(len(systems))]
    with mp.Simulation(systems, 100, 100, seed=11, precision=mp.FP64) as sim:
        sim.run()
        e64 = [sim.estimates(k) for k in range(len(systems))]
    orc = O.run([O.System(L, 1.44, n_paths=P, path_count=min(P, 48)) for L, P in sizes], 100, 100, seed=11)
    for k, (L, _) in enumerate(sizes):
        ref = O.estimates(orc[k], L ** 3, 1.44)
        for key in ("e", "m"):
            z = abs(e32[k][key] - ref[key]) / np.hypot(e32[k][key + "_se"], ref[key + "_se"])
            assert z < 3, (L, key, e32[k][key], ref[key], z)
        assert abs(e32[k]["e"] - e64[k]["e"]) < 1e-4 + 3 * e32[k]["e_se"], (L, e32[k]["e"], e64[k]["e"])


@pytest.mark.parametrize("L", [12, 24])
def test_fp32_mixed_kernel_follows_the_single_size_kernel(L):
    """The mixed-size kernel walks L = 12 and 24 in chunks of 3 planes, the
    kernels compiled for one size in chunks of 6: the per-site arithmetic is
    the same, so the records agree to the rounding of FP32 partial sums."""
    alone = [mp.System(L, 1.2, n_paths=5)]
    a, _ = gpu_records(alone, 3, 4, seed=12)
    b, _ = gpu_records(alone + [mp.System(8, 1.0, n_paths=7)], 3, 4, seed=12)
    np.testing.assert_allclose(b[0][:, FIELDS], a[0][:, FIELDS], rtol=2e-6, atol=2e-7)


def test_in_place_split_schedule_and_spins():
    """The in-place HBM path (FP64 L = 46) through resumable runs: a schedule
    split by a checkpoint equals one run, and the final spins equal the
    oracle's after one sweep."""
    systems = [mp.System(46, 1.1, n_paths=2)]
    with mp.Simulation(systems, 2, 2, seed=3, precision=mp.FP64) as whole:
        whole.run_sweeps(4)
        ref = whole.paths(0)
    with mp.Simulation(systems, 2, 2, seed=3, precision=mp.FP64) as a:
        a.run_sweeps(3)
        blob = a.checkpoint()
    with mp.Simulation(systems, 2, 2, seed=3, precision=mp.FP64) as b:
        b.restore(blob)
        b.run_sweeps(1)
        got = b.paths(0)
    np.testing.assert_allclose(got[:, FIELDS], ref[:, FIELDS], rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(got[:, 17], ref[:, 17])
    with mp.Simulation(systems, 0, 1, seed=3, precision=mp.FP64, keep_spins=True) as sim:
        sim.run()
        spins = [sim.spins(0, p) for p in range(2)]
    _, ospins = O.run([osys(systems[0])], 0, 1, seed=3, want_spins=True)
    for p in range(2):
        np.testing.assert_allclose(spins[p].reshape(-1, 3), ospins[0][p], rtol=0, atol=1e-12)
