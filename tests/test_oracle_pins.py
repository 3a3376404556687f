"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with an
independent implementation (PyTorch's Philox header), a closed form of the
model (open chain, free spins in a field, infinite temperature, two coupled
spins), a limit (low-T equipartition, high-T series), an invariant (energy
bookkeeping, sublattice symmetry, |S| = 1), or a library routine (scipy's
normal probability plot).  Tolerances on Monte Carlo quantities are 4 combined
standard errors plus any stated truncation error of the limit used.
"""
import os
import subprocess

import numpy as np
import pytest
from scipy import stats

import golden
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def langevin(K):
    return 1.0 / np.tanh(K) - 1.0 / K


def zdiff(a, b, se):
    return abs(a - b) / se


# ----------------------------------------------------------------- Philox --
@pytest.fixture(scope="module")
def torch_kat(tmp_path_factory):
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    exe = str(tmp_path_factory.mktemp("kat") / "kat")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I" + inc, "-o", exe,
                           os.path.join(HERE, "philox_torch_kat.cpp")])

    def run(rows):
        inp = "\n".join(" ".join(str(v) for v in r) for r in rows) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return [tuple(int(v) for v in line.split()) for line in out.strip().splitlines()]

    return run


def test_philox_matches_pytorch_header(torch_kat):
    rng = np.random.default_rng(12345)
    rows = [(0, 0, 0, 0, 0, 0), (2**32 - 1,) * 6]
    rows += [tuple(int(v) for v in rng.integers(0, 2**32, 6, dtype=np.uint64)) for _ in range(400)]
    # the counter layout the method uses: (site, sweep, path, tag | system << 8)
    rows += [(i, s, p, (t | (k << 8)), 1, 0) for i in (0, 63, 4095) for s in (0, 1, 3999)
             for p in (0, 255, 4095) for t in (0, 1, 2) for k in (0, 20)]
    ref = torch_kat(rows)
    got = [O.philox(*r) for r in rows]
    assert got == ref


def test_philox_words_uniform():
    w = np.array([O.philox(i, 7, 3, 0, 1, 0) for i in range(20000)], dtype=np.float64)
    u = (w + 0.5) / 2**32
    for k in range(4):
        assert stats.kstest(u[:, k], "uniform").pvalue > 1e-3
    # words of one block are uncorrelated
    c = np.corrcoef(u.T)
    assert np.max(np.abs(c - np.eye(4))) < 0.04


# ------------------------------------------------------- trial move / init --
def test_trial_uniform_on_sphere():
    t = np.array([O.trial(i, 0, 5, 0, 1) for i in range(20000)])
    assert np.max(np.abs(np.linalg.norm(t, axis=1) - 1.0)) < 1e-15
    # uniform on the sphere: cos(theta) ~ U(-1, 1), phi ~ U(-pi, pi)
    assert stats.kstest(t[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-3
    phi = np.arctan2(t[:, 1], t[:, 0])
    assert stats.kstest(phi, "uniform", args=(-np.pi, 2 * np.pi)).pvalue > 1e-3
    assert abs(np.mean(t[:, 0] * t[:, 1])) < 4 * np.sqrt(1 / 15 / t.shape[0])


def test_init_modes():
    s = np.concatenate([O.init(O.SC, 8, p, 0, 1, O.INIT_SPHERE) for p in range(20)])
    assert stats.kstest(s[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-3
    a = np.concatenate([O.init(O.SC, 8, p, 0, 1, O.INIT_ANGLES) for p in range(20)])
    theta = np.arccos(np.clip(a[:, 2], -1, 1))
    assert stats.kstest(theta, "uniform", args=(0, np.pi)).pvalue > 1e-3
    assert abs(np.mean(a[:, 2] ** 2) - 0.5) < 0.01  # <cos^2> = 1/2 for uniform theta
    o = O.init(O.SC, 4, 0, 0, 1, O.INIT_ORDERED)
    assert np.array_equal(o, np.tile([0.0, 0.0, 1.0], (64, 1)))


# ------------------------------------------------------------- energy -----
@pytest.mark.parametrize("L", [2, 4, 6])
def test_energy_ordered_and_neel(L):
    N = L ** 3
    up = np.tile([0.0, 0.0, 1.0], (N, 1))
    # all aligned: every site has 6 bonds of S.S = 1, halved by Eq. (1)
    assert O.energy(O.SC, L, 1.0, 0.0, up) == pytest.approx(-3.0 * N, abs=1e-12)
    assert O.energy(O.SC, L, 1.0, 0.25, up) == pytest.approx(-3.0 * N - 0.25 * N, abs=1e-12)
    idx = np.arange(N)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    sign = np.where((x + y + z) % 2 == 0, 1.0, -1.0)
    neel = up * sign[:, None]
    assert O.energy(O.SC, L, 1.0, 0.0, neel) == pytest.approx(3.0 * N, abs=1e-12)


def test_energy_chain_and_sublattice_symmetry():
    up = np.tile([0.0, 0.0, 1.0], (9, 1))
    assert O.energy(O.CHAIN, 9, 1.0, 0.5, up) == pytest.approx(-8.0 - 4.5, abs=1e-12)
    rng = np.random.default_rng(3)
    for lat, L in ((O.SC, 4), (O.SC, 6), (O.CHAIN, 10)):
        N = L ** 3 if lat == O.SC else L
        s = rng.normal(size=(N, 3))
        s /= np.linalg.norm(s, axis=1, keepdims=True)
        idx = np.arange(N)
        par = (idx % L + (idx // L) % L + idx // (L * L)) % 2 if lat == O.SC else idx % 2
        flipped = s * np.where(par == 1, -1.0, 1.0)[:, None]
        # J -> -J is the same model after flipping one sublattice (Sec. 2.1)
        assert O.energy(lat, L, -1.0, 0.0, flipped) == pytest.approx(O.energy(lat, L, 1.0, 0.0, s), abs=1e-11)


@pytest.mark.parametrize("lat,L", [(O.SC, 2), (O.SC, 4), (O.SC, 6), (O.CHAIN, 7), (O.CHAIN, 8)])
def test_delta_e_equals_energy_difference(lat, L):
    rng = np.random.default_rng(L + 17 * lat)
    N = L ** 3 if lat == O.SC else L
    for _ in range(50):
        s = rng.normal(size=(N, 3))
        s /= np.linalg.norm(s, axis=1, keepdims=True)
        i = int(rng.integers(N))
        t = rng.normal(size=3)
        t /= np.linalg.norm(t)
        J, h = rng.uniform(-2, 2), rng.uniform(-1, 1)
        e0 = O.energy(lat, L, J, h, s)
        s2 = s.copy()
        s2[i] = t
        e1 = O.energy(lat, L, J, h, s2)
        assert O.delta_e(lat, L, J, h, s, i, t) == pytest.approx(e1 - e0, abs=1e-12)


# ------------------------------------------------------- closed forms -----
@pytest.mark.parametrize("T", [1.0, 0.4])
def test_two_spin_detailed_balance(T):
    """Two coupled spins: x = S1.S2 has density proportional to exp(K x) on [-1, 1]."""
    K = 1.0 / T
    rec = O.run([O.System(L=2, T=T, n_paths=20000, lattice=O.CHAIN)], 40, 1)[0]
    x = -2.0 * rec[:, O.REC["fe"]]  # final energy per spin is -J x / 2
    cdf = lambda v: (np.exp(K * v) - np.exp(-K)) / (np.exp(K) - np.exp(-K))  # noqa: E731
    assert stats.kstest(x, cdf).pvalue > 1e-3
    assert zdiff(x.mean(), langevin(K), x.std(ddof=1) / np.sqrt(x.size)) < 4


def test_open_chain_closed_forms():
    """Open chain, h = 0: bond variables are iid, so every moment is closed form."""
    N, T, J = 64, 1.0, 1.0
    K = J / T
    rec = O.run([O.System(L=N, T=T, n_paths=1024, lattice=O.CHAIN)], 300, 700)[0]
    est = O.estimates(rec, N, T)
    ell = langevin(K)
    var_x = 1.0 / K ** 2 - 1.0 / np.sinh(K) ** 2
    e_exact = -J * (N - 1) * ell / N
    assert zdiff(est["e"], e_exact, est["e_se"]) < 4
    var_E = J ** 2 * (N - 1) * var_x
    assert zdiff(est["de_dbeta"], -var_E / N, est["de_dbeta_se"]) < 4
    assert zdiff(est["cv"], var_E / (N * T ** 2), est["cv_se"]) < 4
    d = np.arange(1, N)
    mm = N + 2.0 * np.sum((N - d) * ell ** d)  # <M_tot . M_tot> with <S_i.S_j> = ell^|i-j|
    assert zdiff(est["m2"], mm / N ** 2, est["m2_se"]) < 4
    assert zdiff(est["dmz_dh"], mm / 3.0 / (N * T), est["dmz_dh_se"]) < 4


def test_free_spins_in_field():
    """J = 0: independent spins in a field, <m_z> is the Langevin function."""
    T, h = 0.5, 0.3
    x = h / T
    rec = O.run([O.System(L=4, T=T, J=0.0, h=h, n_paths=512)], 50, 200)[0]
    est = O.estimates(rec, 64, T)
    assert zdiff(est["mz"], langevin(x), est["mz_se"]) < 4
    assert zdiff(est["e"], -h * langevin(x), est["e_se"]) < 4
    dL = 1.0 / x ** 2 - 1.0 / np.sinh(x) ** 2  # L'(x)
    chi_z = dL / T
    assert zdiff(est["dmz_dh"], chi_z, est["dmz_dh_se"]) < 4
    # <e> = -h L(beta h): d<e>/dh = -L(beta h) - beta h L'(beta h), the first term
    # being the field term of e itself
    assert zdiff(est["de_dh"], -langevin(x) - x * dL, est["de_dh_se"]) < 4


def test_infinite_temperature():
    """beta -> 0: every spin is a fresh uniform direction each sweep, so the
    moments are those of N independent unit vectors.  With 3N distinct bonds
    (L = 4), <e^2> = 3N (1/3) / N^2 = 1/N; <|m|^4> = (5N^2 - 2N) / (3N^4),
    hence U_L = 1 - <|m|^4> / (3 <|m|^2>^2) = 4/9 + 2/(9N)."""
    N = 64
    rec = O.run([O.System(L=4, T=1e12, n_paths=512)], 2, 50)[0]
    est = O.estimates(rec, N, 1e12)
    assert est["acc"] == 1.0  # every move is accepted at beta -> 0
    assert zdiff(est["e"], 0.0, est["e_se"]) < 4
    assert zdiff(est["m2"], 1.0 / N, est["m2_se"]) < 4  # <|m|^2> = 1/N for iid spins
    assert zdiff(est["mx"], 0.0, est["mx_se"]) < 4
    assert zdiff(est["e2"], 1.0 / N, est["e2_se"]) < 4
    assert zdiff(est["m4"], (5.0 * N * N - 2.0 * N) / (3.0 * N ** 4), est["m4_se"]) < 4
    assert zdiff(est["binder"], 4.0 / 9.0 + 2.0 / (9.0 * N), est["binder_se"]) < 4


def test_high_temperature_series():
    """Small K: nearest-neighbour correlation is L(K) up to loop terms O(L(K)^3)."""
    T = 20.0
    rec = O.run([O.System(L=4, T=T, n_paths=512)], 20, 100)[0]
    est = O.estimates(rec, 64, T)
    lead = -3.0 * langevin(1.0 / T)
    assert abs(est["e"] - lead) < 4 * est["e_se"] + 12 * langevin(1.0 / T) ** 3 * 3


def test_low_temperature_equipartition():
    """T -> 0 from the ordered start: e = -3J + T (1 - 1/N) + O(T^2), so the
    heat capacity per spin C_V = N beta^2 (<e^2> - <e>^2) tends to 1 - 1/N.

    Two quadratic modes per spin, less the two of a global rotation, each carry
    T/2.  Acceptance is below 1% here, so thermalisation takes ~2000 sweeps.
    """
    L, N = 4, 64
    Ts = [0.03, 0.05]
    recs = O.run([O.System(L=L, T=t, n_paths=256) for t in Ts], 2000, 600,
                 init_mode=O.INIT_ORDERED)
    for r, t in zip(recs, Ts):
        est = O.estimates(r, N, t)
        ratio = (est["e"] + 3.0) / t
        # 4 SE plus an anharmonic allowance of 0.5 T
        assert abs(ratio - (1 - 1 / N)) < 4 * est["e_se"] / t + 0.5 * t
        # the fluctuation estimator of Eq. (cv) gives the same limit
        assert abs(est["cv"] - (1 - 1 / N)) < 4 * est["cv_se"] + t


def test_ordered_start_frozen_at_zero_temperature():
    rec = O.run([O.System(L=4, T=1e-300, n_paths=4)], 0, 3, init_mode=O.INIT_ORDERED)[0]
    assert np.all(rec[:, O.REC["e"]] == -3.0)
    assert np.all(rec[:, O.REC["acc"]] == 0.0)


def test_unit_spins_conserved():
    rec = O.run([O.System(L=4, T=1.5, n_paths=16), O.System(L=16, T=0.7, n_paths=4, lattice=O.CHAIN)], 20, 20)
    for r in rec:
        assert np.all(r[:, O.REC["norm"]] < 5e-16)


def test_random_site_order_agrees_with_checkerboard():
    """Both orders sample the Boltzmann distribution (Sec. 2.2 uses random sites)."""
    sys_ = [O.System(L=4, T=1.5, n_paths=512)]
    a = O.estimates(O.run(sys_, 300, 300, order_mode=O.ORDER_CHECKER)[0], 64, 1.5)
    b = O.estimates(O.run(sys_, 300, 300, order_mode=O.ORDER_RANDOM)[0], 64, 1.5)
    for k in ("e", "m", "m2"):
        assert zdiff(a[k], b[k], np.hypot(a[k + "_se"], b[k + "_se"])) < 4


def test_random_site_order_draws_sites_uniformly():
    """At infinite temperature every move is accepted, so after one sweep of N
    random sites exactly the never-drawn sites keep their initial spin: a
    fraction (1 - 1/N)^N ~ 1/e for uniform draws."""
    L, N, P = 16, 4096, 8
    _, sp = O.run([O.System(L=L, T=1e300, n_paths=P)], 0, 1, order_mode=O.ORDER_RANDOM, want_spins=True)
    kept = 0
    for p in range(P):
        s0 = O.init(O.SC, L, p, 0, 1, O.INIT_SPHERE)
        kept += int(np.sum(np.all(sp[0][p] == s0, axis=1)))
    frac = kept / (N * P)
    expect = (1 - 1 / N) ** N
    assert abs(frac - expect) < 4 * np.sqrt(expect * (1 - expect) / (N * P))


def test_two_start_split_and_convergence():
    """Sec. 4's check: half the paths from the random state, half from the
    ordered state.  The split is exact (each half equals the matching
    single-start run path by path); the halves disagree after one sweep and
    agree once thermalised."""
    s = [O.System(L=4, T=1.0, n_paths=65)]
    two = O.run(s, 0, 1, two_start=True)[0]
    rnd = O.run(s, 0, 1)[0]
    ordd = O.run(s, 0, 1, init_mode=O.INIT_ORDERED)[0]
    np.testing.assert_array_equal(two[:33], rnd[:33])
    np.testing.assert_array_equal(two[33:], ordd[33:])
    early = O.estimates(two, 64, 1.0)
    assert early["e_b"] < early["e_a"] and early["start_z"] > 10
    late = O.estimates(O.run([O.System(L=4, T=1.0, n_paths=512)], 400, 400, two_start=True)[0], 64, 1.0)
    assert late["start_z"] < 4
    assert np.isclose(late["e_a"] * 256 + late["e_b"] * 256, late["e"] * 512)


def _r_critical(n, alpha=1e-3, reps=4000):
    """Lower alpha-quantile of the distribution coefficient for normal samples of size n."""
    rng = np.random.default_rng(2024)
    r = np.array([O.distribution_coefficient(rng.normal(size=n)) for _ in range(reps)])
    return float(np.quantile(r, alpha))


def test_normality_of_path_outputs():
    """Sec. 3, Table 1: per-path outputs are close to normally distributed.

    r (Eq. dist-coefficient) of a sample of n normal values falls below 1 by
    O(1/n), so away from the critical point each r is compared with the 0.1%
    quantile of r over normal samples of the same size: energy deep in the
    ordered phase (T = 0.6) and every output deep in the disordered one
    (T = 2.5).  Near T_C (the paper's T = 1.4..1.6 for L = 10) the magnetisation
    of a finite lattice is not Gaussian (the Binder cumulant is far from 0), so
    there the check is Table 1's own range: r above its smallest entry, 0.9856.
    """
    n = 512
    crit = _r_critical(n)
    assert 0.98 < crit < 0.999
    deep = O.estimates(O.run([O.System(L=10, T=2.5, n_paths=n)], 100, 50)[0], 1000, 2.5)
    for k in ("r_e", "r_mx", "r_my", "r_mz"):
        assert deep[k] > crit, (k, deep[k], crit)
    lo = O.estimates(O.run([O.System(L=10, T=0.6, n_paths=n)], 300, 100,
                           init_mode=O.INIT_ORDERED)[0], 1000, 0.6)
    assert lo["r_e"] > crit, (lo["r_e"], crit)
    table_min = min(v for row in golden.table1().values() for v in row.values() if v is not None)
    assert table_min == 0.9856
    assert lo["r_m"] > table_min
    near = O.estimates(O.run([O.System(L=10, T=1.5, n_paths=n)], 200, 100)[0], 1000, 1.5)
    for k in ("r_e", "r_mx", "r_my", "r_mz"):
        assert near[k] > 0.98, (k, near[k])


# ------------------------------------------------------------- estimates --
def test_distribution_coefficient_against_scipy():
    rng = np.random.default_rng(9)
    q = stats.norm.ppf((np.arange(1, 501) - 0.5) / 500)
    assert O.distribution_coefficient(3.0 + 2.0 * q) == pytest.approx(1.0, abs=1e-12)
    for x in (rng.normal(size=4000), rng.uniform(size=4000), rng.exponential(size=4000)):
        r_scipy = stats.probplot(x, dist="norm")[1][2] ** 2
        assert O.distribution_coefficient(x) == pytest.approx(r_scipy, abs=2e-3)


def test_jackknife_of_mean_is_standard_error():
    from oracle.estimates import _jackknife

    x = np.random.default_rng(4).normal(size=333)
    se = x.std(ddof=1) / np.sqrt(x.size)
    assert _jackknife(lambda m: m["a"], {"a": x}) == pytest.approx(se, rel=1e-10)


# --------------------------------------- derived estimators, two-spin chain --
# Each fluctuation estimator of oracle/estimates.py is fed the exact averages of
# the two-spin chain (tests/two_spin.py: 3-D quadrature, no sampling) and
# compared with what fixes it independently: the central difference of the
# exact <A>(beta, h) for the derivatives (d<e>/dT for C_V), and closed forms for
# chi.  Then one Monte Carlo run of the oracle is compared with the same exact
# values, and planted mistakes (a sign, a power of beta, a moment, a dropped
# term) are shown to fail.
import two_spin  # noqa: E402
import importlib  # noqa: E402

E = importlib.import_module("oracle.estimates")  # the module (the package re-exports a function of that name)

TWO_SPIN_CASES = [(0.7, 1.0, 0.0), (0.7, 1.0, 0.3), (1.3, 1.0, -0.2), (0.5, -1.0, 0.4), (0.9, 0.0, 0.25)]
DERIVATIVES = [("de_dbeta", "e", "beta"), ("dm_dbeta", "m", "beta"), ("dmz_dbeta", "mz", "beta"),
               ("de_dh", "e", "h"), ("dm_dh", "m", "h"), ("dmz_dh", "mz", "h")]


def _exact_estimates(beta, J, h):
    rows = two_spin.record_rows(two_spin.moments(beta, J, h), O.REC, O.NREC)
    return O.estimates(rows, 2, 1.0 / beta)


def _central(obs, beta, J, h, param, step=1e-4):
    if param == "beta":
        p, q = two_spin.moments(beta + step, J, h), two_spin.moments(beta - step, J, h)
    else:
        p, q = two_spin.moments(beta, J, h + step), two_spin.moments(beta, J, h - step)
    return (p[obs] - q[obs]) / (2 * step)


def _check_two_spin_exact(beta, J, h):
    est = _exact_estimates(beta, J, h)
    for name, obs, param in DERIVATIVES:
        fd = _central(obs, beta, J, h, param)
        assert est[name] == pytest.approx(fd, rel=1e-6, abs=1e-8), (name, est[name], fd)
    # C_V per site is d<e>/dT = -beta^2 d<e>/dbeta
    fd_T = -beta ** 2 * _central("e", beta, J, h, "beta")
    assert est["cv"] == pytest.approx(fd_T, rel=1e-6, abs=1e-8), ("cv", est["cv"], fd_T)
    if h == 0.0 and J >= 0.0:
        # chi of Eq. (cv) in closed form; the quadrature's <|m|> is good to ~1e-6
        assert est["chi"] == pytest.approx(two_spin.chi_h0(beta, J), rel=2e-4), ("chi", est["chi"])


@pytest.mark.parametrize("beta,J,h", TWO_SPIN_CASES + [(1.6, 0.0, 0.0), (0.35, 2.0, 0.0)])
def test_derived_estimators_on_exact_two_spin_averages(beta, J, h):
    _check_two_spin_exact(beta, J, h)


def test_chi_closed_forms_of_two_spin_chain():
    """The closed forms the chi pin uses: free pair chi = beta/9; at J > 0 the
    erfi form of <|m|> agrees with direct quadrature of x ~ e^{Kx}."""
    from scipy import integrate

    assert two_spin.chi_h0(1.6, 0.0) == pytest.approx(1.6 / 9.0, rel=1e-15)
    for K in (0.35, 0.7, 1.3, 3.0):
        num, _ = integrate.quad(lambda x: np.sqrt((1 + x) / 2) * np.exp(K * x), -1, 1, epsabs=1e-14)
        den = 2 * np.sinh(K) / K
        assert two_spin.abs_m_h0(K) == pytest.approx(num / den, rel=1e-10)


def test_derived_estimators_on_two_spin_monte_carlo():
    """The oracle's sampled two-spin chain in a field against the exact values,
    every estimate within 4 jackknife standard errors."""
    beta, J, h = 0.7, 1.0, 0.3
    rec = O.run([O.System(L=2, T=1.0 / beta, J=J, h=h, n_paths=4096, lattice=O.CHAIN)], 100, 400, seed=5)[0]
    est = O.estimates(rec, 2, 1.0 / beta)
    exact = _exact_estimates(beta, J, h)
    for k in ("e", "m", "m2", "mz", "chi", "cv", "binder") + tuple(d[0] for d in DERIVATIVES):
        assert zdiff(est[k], exact[k], est[k + "_se"]) < 4, (k, est[k], exact[k], est[k + "_se"])
    # and at h = 0, J = 0.9: chi against its closed form
    rec0 = O.run([O.System(L=2, T=1.0 / beta, J=0.9, n_paths=4096, lattice=O.CHAIN)], 100, 400, seed=6)[0]
    est0 = O.estimates(rec0, 2, 1.0 / beta)
    assert zdiff(est0["chi"], two_spin.chi_h0(beta, 0.9), est0["chi_se"]) < 4


PLANTED = {
    "chi": [lambda m, N, b: N * b ** 2 * (m["m2"] - m["m"] ** 2),       # T^2 for T
            lambda m, N, b: N * b * (m["mz2"] - m["m"] ** 2),           # m_z^2 for |m|^2
            lambda m, N, b: b * (m["m2"] - m["m"] ** 2)],               # N dropped
    "cv": [lambda m, N, b: N * b * (m["e2"] - m["e"] ** 2)],            # T for T^2
    "de_dbeta": [lambda m, N, b: N * (m["e2"] - m["e"] ** 2)],          # sign
    "dm_dbeta": [lambda m, N, b: N * (m["em"] - m["m"] * m["e"]),       # sign
                 lambda m, N, b: -N * (m["emz"] - m["m"] * m["e"])],    # e m_z for e |m|
    "dmz_dbeta": [lambda m, N, b: N * (m["emz"] - m["mz"] * m["e"]),    # sign
                  lambda m, N, b: -N * b * (m["emz"] - m["mz"] * m["e"])],  # stray beta
    "de_dh": [lambda m, N, b: b * N * (m["emz"] - m["e"] * m["mz"]),    # explicit -<m_z> dropped
              lambda m, N, b: b * N * (m["emz"] - m["e"] * m["mz"]) + m["mz"]],  # its sign
    "dm_dh": [lambda m, N, b: N * (m["mmz"] - m["m"] * m["mz"]),        # beta dropped
              lambda m, N, b: b * N * (m["em"] - m["m"] * m["e"])],     # e for m_z
    "dmz_dh": [lambda m, N, b: b * N * (m["mz2"] - m["mz"] * m["m"])],  # |m| for m_z
}


@pytest.mark.parametrize("name,k", [(n, k) for n, fs in PLANTED.items() for k in range(len(fs))])
def test_planted_estimator_mistakes_fail_the_pins(monkeypatch, name, k):
    monkeypatch.setitem(E.DERIVED, name, PLANTED[name][k])
    failed = False
    for case in TWO_SPIN_CASES + [(1.6, 0.0, 0.0), (0.35, 2.0, 0.0)]:
        try:
            _check_two_spin_exact(*case)
        except AssertionError:
            failed = True
            break
    assert failed, f"planted mistake {name}[{k}] passed every pin"
