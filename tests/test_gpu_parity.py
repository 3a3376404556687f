"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars (FP64 form): Philox words bit-identical; spins within 1e-12 of the
oracle over the first 10 sweeps; per-path records within 1e-10 relative
(summation order differs); estimates of the reduction kernel within 1e-9 of
the oracle's estimates on the same records.  FP32 form: ensemble means within
3 combined standard errors of the oracle, per-path outputs after one sweep of
the full-size launch within 1e-5 (FP32 rounding can flip a borderline accept,
so a small fraction of sampled paths may differ and is counted).
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1305_6758_gb300 as mp  # noqa: E402

RECORD_FIELDS = list(range(17))  # means and final state


def osys(s, **kw):
    return O.System(L=s.L, T=s.T, J=s.J, h=s.h, n_paths=s.n_paths, lattice=s.lattice, **kw)


def run_gpu(systems, n_therm, n_meas, seed=1, **kw):
    with mp.Simulation(systems, n_therm, n_meas, seed=seed, **kw) as sim:
        sim.run()
        recs = [sim.paths(k) for k in range(len(systems))]
        ests = [sim.estimates(k) for k in range(len(systems))]
        spins = None
        if kw.get("keep_spins"):
            spins = [np.stack([sim.spins(k, p) for p in range(s.n_paths)]) for k, s in enumerate(systems)]
    return recs, ests, spins


# ------------------------------------------------------------------ Philox --
def test_philox_bit_identical():
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2**32, size=(3000, 4), dtype=np.uint64).astype(np.uint32)
    # the counters the sweep uses: (site, sweep, path, tag | system << 8)
    lay = np.array([(i, s, p, t | (k << 8)) for i in (0, 1, 4095) for s in (0, 1999, 3999)
                    for p in (0, 4095) for t in (0, 1) for k in (0, 20)], dtype=np.uint32)
    ctr = np.concatenate([ctr, lay, np.full((1, 4), 2**32 - 1, dtype=np.uint32)])
    for seed in (1, 0xDEADBEEFCAFEF00D):
        got = mp.philox(ctr, seed)
        k0, k1 = seed & 0xFFFFFFFF, seed >> 32
        ref = np.array([O.philox(*map(int, c), k0, k1) for c in ctr], dtype=np.uint32)
        assert np.array_equal(got, ref)


# ------------------------------------------------------- FP64 trajectories --
def test_fp64_spins_first_ten_sweeps_plain_config():
    """Simple cubic L=4, J=1, h=0, T=1.5, 256 paths, seed 1: spins after sweeps 1..10."""
    systems = [mp.System(4, 1.5, n_paths=256)]
    worst = 0.0
    for k in range(1, 11):
        _, _, spins = run_gpu(systems, 0, k, precision=mp.FP64, keep_spins=True)
        _, ref = O.run([osys(systems[0])], 0, k, want_spins=True)
        d = np.abs(spins[0] - ref[0]).max()
        worst = max(worst, d)
        assert d < 1e-12, f"sweep {k}: max spin difference {d}"
    print("max spin difference over 10 sweeps", worst)


def test_fp64_records_and_estimates_plain_config():
    """The full plain-method configuration: 256 paths x (1000 + 1000) sweeps, FP64."""
    systems = [mp.System(4, 1.5, n_paths=256)]
    recs, ests, _ = run_gpu(systems, 1000, 1000, precision=mp.FP64)
    ref = O.run([osys(systems[0])], 1000, 1000)[0]
    np.testing.assert_allclose(recs[0][:, RECORD_FIELDS], ref[:, RECORD_FIELDS], rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(recs[0][:, 17], ref[:, 17], rtol=0, atol=0)  # acceptance counts exact
    # the reduction kernel against the oracle's estimates of the same records
    oest = O.estimates(recs[0], 64, 1.5)
    for k, v in oest.items():
        if k in ests[0]:
            assert ests[0][k] == pytest.approx(v, rel=1e-9, abs=1e-12), k


@pytest.mark.parametrize("name,systems,init", [
    ("L2-degenerate", [mp.System(2, 0.8, h=0.1, n_paths=64)], mp.INIT_SPHERE),
    ("chain-odd", [mp.System(7, 0.7, J=-1.0, n_paths=33, lattice=mp.CHAIN)], mp.INIT_SPHERE),
    ("chain-two", [mp.System(2, 0.5, n_paths=40, lattice=mp.CHAIN)], mp.INIT_ANGLES),
    ("uneven-batch", [mp.System(8, 1.2, n_paths=37), mp.System(4, 2.0, h=-0.2, n_paths=5),
                      mp.System(10, 1.44, n_paths=3), mp.System(64, 1.0, n_paths=70, lattice=mp.CHAIN),
                      mp.System(12, 0.9, n_paths=2)], mp.INIT_SPHERE),
    ("ordered-start", [mp.System(6, 0.3, n_paths=9)], mp.INIT_ORDERED),
    ("single-path", [mp.System(16, 1.0, n_paths=1)], mp.INIT_SPHERE),
])
def test_fp64_edge_cases(name, systems, init):
    recs, ests, _ = run_gpu(systems, 3, 4, seed=11, precision=mp.FP64, init_mode=init)
    refs = O.run([osys(s) for s in systems], 3, 4, seed=11, init_mode=init)
    for s, g, r, e in zip(systems, recs, refs, ests):
        np.testing.assert_allclose(g[:, RECORD_FIELDS], r[:, RECORD_FIELDS], rtol=1e-10, atol=1e-13)
        assert e["n_paths"] == s.n_paths
        if s.n_paths == 1:
            assert np.isnan(e["e_se"]) and np.isnan(e["chi_se"])


def test_fp64_largest_shared_memory_lattice():
    """L=20 (192 KB of FP64 spins per path), a few paths, a few sweeps."""
    systems = [mp.System(20, 1.3, n_paths=3)]
    recs, _, _ = run_gpu(systems, 1, 2, seed=2, precision=mp.FP64)
    ref = O.run([osys(systems[0])], 1, 2, seed=2)[0]
    np.testing.assert_allclose(recs[0][:, RECORD_FIELDS], ref[:, RECORD_FIELDS], rtol=1e-10, atol=1e-13)


# ----------------------------------------------------------------- FP32 ----
def test_fp32_plain_config_ensemble():
    systems = [mp.System(4, 1.5, n_paths=256)]
    _, ests, _ = run_gpu(systems, 1000, 1000)
    ref = O.estimates(O.run([osys(systems[0])], 1000, 1000)[0], 64, 1.5)
    for k in ("e", "m", "m2", "mx", "mz"):
        z = abs(ests[0][k] - ref[k]) / np.hypot(ests[0][k + "_se"], ref[k + "_se"])
        assert z < 3, (k, ests[0][k], ref[k], z)
    assert ests[0]["norm_max"] < 2e-6


FULL_T = [0.5 + 0.1 * k for k in range(21)]


@pytest.mark.parametrize("precision,tol", [(mp.FP32, 1e-5), (mp.FP64, 1e-12)])
def test_full_size_launch_first_sweep(precision, tol):
    """The benchmark's launch (L=16, 21 temperatures x 4096 paths, same plan)
    after one sweep: sampled paths of every system against the oracle, path by path."""
    systems = [mp.System(16, T, n_paths=4096) for T in FULL_T]
    with mp.Simulation(systems, 0, 1, seed=1, precision=precision) as sim:
        sim.run()
        recs = [sim.paths(k) for k in range(len(systems))]
    bad, total = 0, 0
    for begin, count in ((0, 2), (2047, 1), (4094, 2)):
        refs = O.run([O.System(16, T, n_paths=4096, path_begin=begin, path_count=count) for T in FULL_T],
                     0, 1)
        for k in range(len(FULL_T)):
            for j in range(count):
                g, r = recs[k][begin + j], refs[k][j]
                total += 1
                bad += int(np.max(np.abs(g[RECORD_FIELDS] - r[RECORD_FIELDS])) > tol)
    limit = 0 if precision == mp.FP64 else max(1, total // 50)
    assert bad <= limit, f"{bad} of {total} sampled paths differ beyond {tol}"


def test_fp32_against_fp64_and_oracle_l16():
    """L=16 at three temperatures of the benchmark range, shortened runs:
    FP32 GPU, FP64 GPU and the oracle agree within 3 combined SE."""
    Ts = [0.5, 1.5, 2.5]
    systems = [mp.System(16, T, n_paths=2048) for T in Ts]
    _, e32, _ = run_gpu(systems, 150, 150, seed=7)
    _, e64, _ = run_gpu(systems, 150, 150, seed=7, precision=mp.FP64)
    orc = O.run([O.System(16, T, n_paths=2048, path_count=64) for T in Ts], 150, 150, seed=7)
    for k, T in enumerate(Ts):
        ref = O.estimates(orc[k], 4096, T)
        for key in ("e", "m"):
            for est in (e32[k], e64[k]):
                z = abs(est[key] - ref[key]) / np.hypot(est[key + "_se"], ref[key + "_se"])
                assert z < 3, (T, key, est[key], ref[key], z)
        # same seed: FP32 and FP64 paths start identical, so their energies are close
        assert abs(e32[k]["e"] - e64[k]["e"]) < 1e-4 + 3 * e32[k]["e_se"]


def test_open_chain_closed_form_and_backward():
    """Open chain of 64 spins, h = 0: energy, d<e>/dbeta and d<m_z>/dh closed forms;
    the backward kernel equals the fluctuation estimators of the reduction."""
    N, T = 64, 1.0
    K = 1.0 / T
    ell = 1 / np.tanh(K) - 1 / K
    systems = [mp.System(N, T, n_paths=4096, lattice=mp.CHAIN)]
    with mp.Simulation(systems, 200, 800, seed=5) as sim:
        sim.run()
        est = sim.estimates(0)
        gb, gh = sim.backward([1.0], [0.0])
        gb2, gh2 = sim.backward([0.0], [1.0])
    e_exact = -(N - 1) * ell / N
    assert abs(est["e"] - e_exact) < 4 * est["e_se"]
    var_E = (N - 1) * (1 / K**2 - 1 / np.sinh(K) ** 2)
    assert abs(est["de_dbeta"] - (-var_E / N)) < 4 * est["de_dbeta_se"]
    d = np.arange(1, N)
    mm = N + 2.0 * np.sum((N - d) * ell ** d)
    assert abs(est["dmz_dh"] - mm / 3 / (N * T)) < 4 * est["dmz_dh_se"]
    assert gb.item() == pytest.approx(est["de_dbeta"], rel=1e-9)
    assert gh.item() == pytest.approx(est["de_dh"], rel=1e-9, abs=1e-12)
    assert gb2.item() == pytest.approx(est["dm_dbeta"], rel=1e-9)
    assert gh2.item() == pytest.approx(est["dm_dh"], rel=1e-9, abs=1e-12)


def test_field_derivatives_reduction_and_backward():
    """h != 0: the reduction's field and temperature derivatives (d<e>/dh with
    the -<m_z> of e's own field term) equal the oracle's estimates of the same
    records, the backward kernel equals them, and for free spins (J = 0)
    d<e>/dh = -L(beta h) - beta h L'(beta h) within 4 SE."""
    systems = [mp.System(4, 1.0, h=0.3, n_paths=512), mp.System(4, 0.5, J=0.0, h=0.3, n_paths=512)]
    with mp.Simulation(systems, 100, 400, seed=9, precision=mp.FP64) as sim:
        sim.run()
        recs = [sim.paths(k) for k in range(2)]
        ests = [sim.estimates(k) for k in range(2)]
        gb, gh = sim.backward([1.0, 1.0], [0.0, 0.0])
        gb2, gh2 = sim.backward([0.0, 0.0], [1.0, 1.0])
    for k, s in enumerate(systems):
        oest = O.estimates(recs[k], 64, s.T)
        for key in ("chi", "cv", "binder", "de_dbeta", "dm_dbeta", "dmz_dbeta", "de_dh", "dm_dh", "dmz_dh"):
            assert ests[k][key] == pytest.approx(oest[key], rel=1e-9, abs=1e-12), key
            assert ests[k][key + "_se"] == pytest.approx(oest[key + "_se"], rel=1e-7, abs=1e-12), key
        assert gb[k].item() == pytest.approx(ests[k]["de_dbeta"], rel=1e-9)
        assert gh[k].item() == pytest.approx(ests[k]["de_dh"], rel=1e-9)
        assert gb2[k].item() == pytest.approx(ests[k]["dm_dbeta"], rel=1e-9)
        assert gh2[k].item() == pytest.approx(ests[k]["dm_dh"], rel=1e-9)
    x = 0.3 / 0.5
    lang = 1 / np.tanh(x) - 1 / x
    closed = -lang - x * (1 / x**2 - 1 / np.sinh(x) ** 2)
    assert abs(ests[1]["de_dh"] - closed) < 4 * ests[1]["de_dh_se"], (ests[1]["de_dh"], closed)


def test_distribution_coefficient_beyond_shared_memory_sort():
    """Eq. (dist-coefficient) for systems of more than 16384 paths (sorted in a
    device buffer instead of shared memory) equals the oracle's r of the same
    records; a small system of the same batch keeps the shared-memory sort; the
    estimates carry the run's device time."""
    systems = [mp.System(4, 1.5, n_paths=20000), mp.System(4, 0.9, n_paths=700)]
    with mp.Simulation(systems, 10, 20, seed=13, precision=mp.FP64) as sim:
        sim.run()
        recs = [sim.paths(k) for k in range(2)]
        ests = [sim.estimates(k) for k in range(2)]
        sweep_ms, reduce_ms = sim.timing()
    for k, s in enumerate(systems):
        oest = O.estimates(recs[k], 64, s.T)
        for key in ("r_e", "r_m", "r_mx", "r_my", "r_mz", "r_amz"):
            assert np.isfinite(ests[k][key])
            assert ests[k][key] == pytest.approx(oest[key], rel=1e-9, abs=1e-12), (k, key)
        assert ests[k]["elapsed_s"] == pytest.approx((sweep_ms + reduce_ms) / 1e3, rel=1e-3)


# ---------------------------------------------------------------- errors ---
def test_status_codes():
    with pytest.raises(mp.MPError) as ei:
        mp.Simulation([mp.System(5, 1.0)], 1, 1)
    assert ei.value.status == mp.MP_EINVAL
    with pytest.raises(mp.MPError) as ei:
        mp.Simulation([mp.System(4, 1.0)], 1, 0)
    assert ei.value.status == mp.MP_EINVAL
    with pytest.raises(mp.MPError) as ei:  # L = 32 runs on two-CTA clusters of 512 threads
        mp.Simulation([mp.System(32, 1.0)], 1, 1, cta_threads=256)
    assert ei.value.status == mp.MP_EINVAL
    sim = mp.Simulation([mp.System(4, 1.0, n_paths=4)], 1, 1)
    with pytest.raises(mp.MPError) as ei:
        sim.estimates(0)
    assert ei.value.status == mp.MP_ESTATE
    with pytest.raises(mp.MPError) as ei:
        sim.spins(0, 0)
    assert ei.value.status == mp.MP_ESTATE
    sim.run()
    with pytest.raises(mp.MPError) as ei:
        sim.estimates(3)
    assert ei.value.status == mp.MP_EINVAL
    sim.close()


def test_rerun_and_seed():
    systems = [mp.System(6, 1.2, n_paths=64)]
    with mp.Simulation(systems, 10, 10, seed=1) as sim:
        sim.run()
        a = sim.paths(0)
        sim.run()
        b = sim.paths(0)
        sim.set_seed(2)
        sim.run()
        c = sim.paths(0)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


# ----------------------------------------------------- thread layouts -------
@pytest.mark.parametrize("L,tp", [
    (8, 32),    # one whole column of 8 planes per thread
    (8, 64),    # columns cut in 2 segments
    (8, 96),    # 8 segments of 1 plane, dealt out in rounds (some threads idle in the last)
    (8, 128),   # 4 segments of 2 planes
    (8, 160),   # uneven rounds
    (12, 288),  # 4 segments of 3 planes
    (12, 96),   # 4 segments of 3 planes over 3 rounds
    (16, 128),  # the benchmark layout: one column per thread
    (16, 256),
    (20, 160),  # 4 segments of 5 planes over 5 rounds
])
def test_fp64_every_walk_layout_matches_oracle(L, tp):
    """Each thread-to-site layout of the shared-memory sweep (column
    segments that carry z and x neighbours from site to site, dealt out to
    the threads in even or uneven rounds) gives the oracle's per-path records."""
    systems = [mp.System(L, 1.1, h=0.03, n_paths=5)]
    recs, _, _ = run_gpu(systems, 2, 3, seed=8, precision=mp.FP64, threads_per_path=tp)
    ref = O.run([osys(systems[0])], 2, 3, seed=8)[0]
    np.testing.assert_allclose(recs[0][:, RECORD_FIELDS], ref[:, RECORD_FIELDS], rtol=1e-10, atol=1e-13)
    np.testing.assert_array_equal(recs[0][:, 17], ref[:, 17])
    with mp.Simulation(systems, 1, 1, precision=mp.FP64, threads_per_path=tp) as sim:
        assert sim.system_plan(0)["threads_per_path"] == tp


def test_fp32_trajectories_do_not_depend_on_the_layout():
    """FP32, L=16: column segments of 16, 8 and 4 planes, uneven rounds and
    paths of one warp give the same records (the same arithmetic per site in
    the same order)."""
    systems = [mp.System(16, 1.3, n_paths=6)]
    base = None
    for tp in (128, 256, 512, 96, 32):
        recs, _, _ = run_gpu(systems, 3, 5, seed=9, threads_per_path=tp)
        if base is None:
            base = recs[0]
        else:
            np.testing.assert_allclose(recs[0][:, RECORD_FIELDS], base[:, RECORD_FIELDS], rtol=2e-6, atol=2e-7)
